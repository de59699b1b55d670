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

#include <stdint.h>

#include "fv.h"

#ifdef __cplusplus
extern "C" {
#endif

int fv_host_xface(const double* model, const double* qm, const double* qp, double* Dm, double* Dp);
int fv_host_yface(const double* model, const double* qm, const double* qp, double* Dm, double* Dp);
/* fv_host_xface_or: D-, D+ at an x face with the conservative Osher-Romberg
 * viscosity of Eq. (OR_cons) (Romberg nodes on the segment path, b4x = u
 * Delta alpha on each sub-segment, Romberg average of u on the face);
 * arguments as fv_host_xface. */
int fv_host_xface_or(const double* model, const double* qm, const double* qp, double* Dm,
                     double* Dp);

/* fv_host_face_f32: D-, D+ of an x face (which = 0, Gauss-Legendre Osher) or a
 * y face (which = 1, well-balanced Osher-Romberg with the alpha p jump of the
 * two states) in FP32: the states are rounded to float and the float solver
 * runs either in the paired form the FP32 step kernels use (paired = 1, two
 * quadrature nodes or Romberg terms per float2 operation) or in the scalar
 * form (paired = 0).  model as for fv_host_xface; outputs widened to double.
 * Returns 1 for a null pointer or another `which`, else 0. */
int fv_host_face_f32(int which, const double* model, const double* qm, const double* qp,
                     int paired, double* Dm, double* Dp);
/* fv_host_yface_o1: D-, D+ of the first-order y face (Sections 3.2-3.3)
 * between the centre of a lower cell at height ya above the level and an upper
 * one dy higher: fa, fb = fluctuations (alpha rho - alpha^E rho^E, alpha rho u,
 * alpha rho v, alpha - alpha^E), aEa, aEb = alpha^E; rho^E and p^E at the
 * quarter heights as the kernels' tables hold them.  Returns 0, or 1 on a null
 * pointer. */
int fv_host_yface_o1(const double* model, const double* fa, double aEa, const double* fb,
                     double aEb, double ya, double dy, double* Dm, double* Dp);

/* Algorithmic operation count of one cell-update of the kernels (one
 * second-order reconstruction with predictor, one x face, one y face, the
 * interior integral of Eq. (Scheme), the update and the epilogue), obtained by
 * running the kernels' per-cell arithmetic on a counting type on the host:
 * out[0..4] = additions, multiplications, divisions, square roots,
 * comparisons.  Returns 0, or 1 on a null pointer. */
int fv_host_cell_ops(double* out);

/* The same count for a cell that the order switch of Section 3.4 (alpha <=
 * 10 eps) advances at first order: its reconstruction is its own fluctuation
 * (the equilibrium products only); faces, interior integral, update and
 * epilogue as above.  Returns 0, or 1 on a null pointer. */
int fv_host_cell_ops_first_order(double* out);

/* Forward value and reverse-mode derivative of one per-face or per-cell
 * function of the kernels (the building blocks of fv_adjoint), on the host.
 * which = 0: x face, in = qm[4], qp[4], out = D-[4], D+[4];
 *         1: y face (dap = c2 (dq0 - rho0 dq3)), same layout;
 *         2: reconstruction of Section 3.4 (limiter, order switch, predictor,
 *            face states, admissibility fallback): in = Qf[4], fW[4], fE[4],
 *            fS[4], fN[4], mx[4], mn[4], alpha^E (29); out = face states
 *            W, E, S, N [16], centre [4], limited alpha slopes [2];
 *         3: interior integral: in = fW[4], fE[4], fS[4], fN[4], centre[4],
 *            alpha^E, dax, day (23); out = Ix[4], Iy[4].
 * k (which 2, 3) = {dx, dy, dt, rhoE_c, rhoE_S, rhoE_N}; the equilibrium
 * masses are alpha^E rhoE.  If lout is not null, lin receives d<lout, out>/d in
 * with every branch held as at `in`.  Returns 0, or 1 on a bad argument. */
int fv_host_adj_check(int which, const double* model, const double* k, const double* in,
                      const double* lout, double* out, double* lin);

/* One reverse step of fv_adjoint on the host: lam_out = lam + (dQ^{n+1}/dQ^n)^T
 * lam for the step with levels K (nx int32) and time step dt held fixed,
 * through the same per-cell and per-face code as the adjoint kernels, in the
 * arithmetic of prec (FV_FP64: full state in double; FV_FP32_DEV: q rounded
 * to the float deviation form relative to K, float arithmetic).  grid, eos,
 * side, solid (ny*nx) as for fv_create; q (full state), lam, lam_out: 4 planes
 * of ny*nx doubles (host).  Returns 0, or 1 on a bad argument. */
int fv_host_adjoint_step(const fv_grid* grid, const fv_eos* eos, const int32_t side[4],
                         const uint8_t* solid, const double* q, const int32_t* K, double dt,
                         const double* lam, double* lam_out, int prec);

/* Obstacle-height part of one reverse step on the host, through the same
 * per-cell code as fv_adjoint's kernel: out[k] = lam . dQ^{n+1}/dtheta_k at
 * theta = 0+, where raising obstacle k by theta dy gives its top cells
 * (height_id as in fv_adjoint_spec) the capacity 1 - theta (the extension
 * documented with fv_adjoint_spec).  Arguments as fv_host_adjoint_step; lam is
 * the adjoint of Q^{n+1} in the storage form of prec (FV_FP64: the full
 * state; FV_FP32_DEV: (alpha rho - alpha rho^E, alpha rho u, alpha rho v,
 * alpha) with rho^E from the levels K); out: nheights doubles.  Returns 0, or
 * 1 on a bad argument. */
int fv_host_height_step(const fv_grid* grid, const fv_eos* eos, const int32_t side[4],
                        const uint8_t* solid, const double* q, const int32_t* K, double dt,
                        const double* lam, const int32_t* height_id, int nheights, double* out,
                        int prec);

#ifdef __cplusplus
}
#endif

#endif /* FV_MODEL_HOST_H */
