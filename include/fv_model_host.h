/*
 * fv_model_host.h -- host evaluation of the face fluctuations that libfv's
 * kernels use, exported for verification without a GPU.
 *
 * fv_host_xface: D-, D+ of Eq. (FIrstOrderDgeneric_x) at an x face with the
 *   Osher viscosity of Eq. (OsherMatrixFormal_approx) (3-point Gauss-Legendre
 *   on the segment path) and b4x = u_bar Delta alpha, u_bar the same
 *   quadrature of u along the path.
 * fv_host_yface: D-, D+ of Eq. (FIrstOrderDgeneric_y) at a y face with the
 *   well-balanced Osher-Romberg viscosity of Eq. (ViscosityOR), both states at
 *   the same height (second order).
 *
 * Arguments: qm, qp = (alpha rho, alpha rho u, alpha rho v, alpha) on the -/+
 * side (host arrays of 4 doubles); model = {rho0, k0, gamma, g, eps_gas} with
 * gamma = 1; Dm, Dp receive 4 doubles each.  Same arithmetic as the device
 * code (compiled for the host); no device memory is touched.  Returns 0, or 1
 * on a null pointer.
 */
#ifndef FV_MODEL_HOST_H
#define FV_MODEL_HOST_H

#ifdef __cplusplus
extern "C" {
#endif

int fv_host_xface(const double* model, const double* qm, const double* qp, double* Dm, double* Dp);
int fv_host_yface(const double* model, const double* qm, const double* qp, double* Dm, double* Dp);

/* Algorithmic operation count of one cell-update of the kernels (one
 * second-order reconstruction with predictor, one x face, one y face, the
 * interior integral of Eq. (Scheme), the update and the epilogue), obtained by
 * running the kernels' per-cell arithmetic on a counting type on the host:
 * out[0..4] = additions, multiplications, divisions, square roots,
 * comparisons.  Returns 0, or 1 on a null pointer. */
int fv_host_cell_ops(double* out);

#ifdef __cplusplus
}
#endif

#endif /* FV_MODEL_HOST_H */
