// Bounds checks of the bounds-checked build (libfk_checked.so, compiled with FK_CHECKED),
// the stand-in for a memory checker: the data-dependent indices of the spreading kernels
// (cells named by partition records, list links, grid nodes, bucket slots) are tested
// before the access.  A failed test sets the internal-error flag, which the call returns
// as FK_EINTERNAL, and the access is skipped; there is no trap and no assert.  In the
// normal build the tests compile to nothing.
#pragma once

namespace fk {

#ifdef FK_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// `ok` in the checked build (setting the flag when it fails), true otherwise
__device__ __forceinline__ bool fk_check(bool ok, unsigned* flags) {
  if (!kChecked) return true;
  if (!ok) atomicOr(flags, 4u /* FLAG_INTERNAL */);
  return ok;
}

}  // namespace fk
