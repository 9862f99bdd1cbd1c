// sgn_spectral_df_rhs.cu - the double-float right-hand side of precision 3
// (its transforms, products and K spectra); the templates are in
// sgn_spectral.cuh.
#define SGN_SPECTRAL_DF_RHS
#include "sgn_spectral.cuh"

namespace sgn {

template cudaError_t launch_rhs<dfl, double>(const Geom&, const Tables<dfl>&, const Tables<double>&,
                                             cpx<double>* const*, const cpx<double>*, const dfl*,
                                             const dfl*, cpx<dfl>* const*, cpx<double>* const*,
                                             cpx<double>* const*, cpx<double>* const*, cpx<double>*,
                                             const RkArgs&, const Exec&);

}  // namespace sgn
