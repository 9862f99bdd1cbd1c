// sgn_spectral_f32.cu - the FP32 spectral passes of the mixed-precision paths:
// the inner GMRES matvec and the right-hand side (its nonlinear part; the RK
// update adds the linear part in FP64); the templates are in sgn_spectral.cuh.
#include "sgn_spectral.cuh"

namespace sgn {

template void init_kernel_attributes<float>();
template cudaError_t launch_matvec<float>(const Geom&, const Tables<float>&, const cpx<float>*, const float*,
                                          const float*, cpx<float>*, cpx<float>* const*, bool, const Exec&,
                                          const int*, size_t, const MvTma*);
template cudaError_t launch_rhs<float, double>(const Geom&, const Tables<float>&, const Tables<double>&,
                                               cpx<double>* const*, const cpx<double>*, const float*,
                                               const float*, cpx<float>* const*, cpx<double>* const*,
                                               cpx<double>* const*, cpx<double>* const*, cpx<double>*,
                                               const RkArgs&, const Exec&);

}  // namespace sgn
