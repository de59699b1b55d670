// Host instantiation of the device face solvers (include/fv_model_host.h).
#include <cmath>

#include "fv_model.cuh"
#include "fv_model_host.h"

namespace {
fv::Phys<double> phys(const double* model) {
  fv::Phys<double> P;
  P.rho0 = model[0];
  P.k0 = model[1];
  P.g = model[3];
  P.c2 = model[1] / model[0];
  P.c = std::sqrt(P.c2);
  P.inv_c = 1.0 / P.c;
  P.kappa = model[3] * model[0] / model[1];
  return P;
}
}  // namespace

extern "C" int fv_host_xface(const double* model, const double* qm, const double* qp, double* Dm,
                             double* Dp) {
  if (!model || !qm || !qp || !Dm || !Dp) return 1;
  const double dq[4] = {qp[0] - qm[0], qp[1] - qm[1], qp[2] - qm[2], qp[3] - qm[3]};
  fv::xface<double>(qm, qp, dq, phys(model), Dm, Dp);
  return 0;
}

extern "C" int fv_host_yface(const double* model, const double* qm, const double* qp, double* Dm,
                             double* Dp) {
  if (!model || !qm || !qp || !Dm || !Dp) return 1;
  const double dq[4] = {qp[0] - qm[0], qp[1] - qm[1], qp[2] - qm[2], qp[3] - qm[3]};
  fv::yface<double>(qm, qp, dq, phys(model), Dm, Dp);
  return 0;
}
