// sgn_spectral.cu - the FP64 spectral passes (the paper's method) and the host
// code the passes share (launch shapes, tensor maps); the templates are in
// sgn_spectral.cuh.
#define SGN_SPECTRAL_COMMON
#include "sgn_spectral.cuh"

namespace sgn {

SGN_INST(double)

template cudaError_t launch_rhs<double, double>(const Geom&, const Tables<double>&, const Tables<double>&,
                                                cpx<double>* const*, const cpx<double>*, const double*,
                                                const double*, cpx<double>* const*, cpx<double>* const*,
                                                cpx<double>* const*, cpx<double>* const*, cpx<double>*,
                                                const RkArgs&, const Exec&);

}  // namespace sgn
