// Mixed-length apply kernels (fft_mixed.cuh) for double: the launchers that
// apply_kernels.cuh declares, instantiated for every pass kind.
#define FRAC_MX_TU
#define FRAC_MX_PASSES_INLINE
#include "apply_kernels.cuh"

namespace frac {

template int launch_conv1d_mx<double, false>(const MxLine&, const double*, double*, int64_t, int64_t, const double*, cudaStream_t);
template int launch_conv1d_mx<double, true>(const MxLine&, const double*, double*, int64_t, int64_t, const double*, cudaStream_t);
#define FRAC_ROWS(K)                                                                                                \
  template int launch_rows_fwd_mx<double, K>(const MxLine&, const void*, void*, int64_t, int64_t, int64_t, int,       \
                                          const CgArgs&, cudaStream_t);
FRAC_ROWS(RF_PLAIN)
FRAC_ROWS(RF_CG)
FRAC_ROWS(RF_ODD)
#undef FRAC_ROWS
#define FRAC_ROWS(K)                                                                                                \
  template int launch_rows_inv_mx<double, K>(const MxLine&, const void*, void*, int64_t, int64_t, int64_t, int,       \
                                          const CgArgs&, cudaStream_t);
FRAC_ROWS(RI_PLAIN)
FRAC_ROWS(RI_CG)
FRAC_ROWS(RI_ODD)
FRAC_ROWS(RI_ODD_CG)
#undef FRAC_ROWS
#define FRAC_COLS(MODE, ODD)                                                                                          \
  template int launch_cols_mx<double, MODE, ODD>(const MxLine&, const void*, void*, const ColArgs&, int64_t, const double*, \
                                              const CGState*, cudaStream_t);
FRAC_COLS(SYM2, false)
FRAC_COLS(YFWD, false)
FRAC_COLS(ZSYM, false)
FRAC_COLS(YINV, false)
FRAC_COLS(SYM2, true)
FRAC_COLS(YFWD, true)
FRAC_COLS(ZSYM, true)
FRAC_COLS(YINV, true)
#undef FRAC_COLS

}  // namespace frac
