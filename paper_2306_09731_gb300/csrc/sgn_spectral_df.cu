// sgn_spectral_df.cu - the double-float spectral passes of precisions 2 and 3:
// the refinement residual's matvec, the coefficients and the state
// conversions (precision 3's right-hand side is in sgn_spectral_df_rhs.cu);
// the templates are in sgn_spectral.cuh.
#define SGN_SPECTRAL_DF
#include "sgn_spectral.cuh"

namespace sgn {

template cudaError_t launch_matvec_io<dfl, double>(const Geom&, const Tables<dfl>&, const cpx<double>*,
                                                   const dfl*, const dfl*, cpx<double>*, cpx<dfl>* const*, bool,
                                                   const Exec&, const int*, size_t);
template cudaError_t launch_y_inv64<dfl>(const Geom&, const Tables<dfl>&, const cpx<double>*, cpx<dfl>*,
                                         const Exec&);
template cudaError_t launch_y_fwd64<dfl>(const Geom&, const Tables<dfl>&, const cpx<dfl>*, cpx<double>*,
                                         const Exec&);
template cudaError_t launch_x_r2c<dfl>(const Geom&, const Tables<dfl>&, const double* const*, int,
                                       cpx<dfl>* const*, const Exec&);
template cudaError_t launch_x_c2r<dfl>(const Geom&, const Tables<dfl>&, const cpx<dfl>* const*, const int*, int,
                                       double* const*, double, const Exec&);
template cudaError_t launch_coef_x<dfl>(const Geom&, const Tables<dfl>&, const cpx<dfl>*, dfl*, dfl*, dfl*, int*,
                                        const CoefCopy&, const Exec&);
template cudaError_t launch_coef_phys<dfl>(const Geom&, const double*, dfl*, dfl*, dfl*, int*, const CoefCopy&,
                                           const Exec&);

}  // namespace sgn
