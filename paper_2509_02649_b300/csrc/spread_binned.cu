// Binned register-accumulation spreading (placeholder until the kernel lands).
#include "fk_internal.cuh"

namespace fk {

bool spread_binned_supported(const EsPlan& p, int n_ch) {
  (void)p;
  (void)n_ch;
  return false;
}

fk_status spread_binned(const EsPlan& p, int64_t n, const float* x, const float* y, int n_y, bool with_ones,
                        double* grid, unsigned* flags, cudaStream_t st, Scratch& scratch) {
  (void)p; (void)n; (void)x; (void)y; (void)n_y; (void)with_ones; (void)grid; (void)flags; (void)st; (void)scratch;
  return set_error(FK_EINVAL, "binned spreading not built");
}

}  // namespace fk
