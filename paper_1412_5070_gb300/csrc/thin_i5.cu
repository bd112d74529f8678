// thin_i5.cu -- instances of the thin contraction for I5 quartets of total order L <= 2, and the
// dispatch over all thin instances.
#include "thin.cuh"

namespace f12k {

ThinKernel thin_kernel_i5(int key) {
#define F12_THIN(K) \
  case K: return thin_entry<K, true>();
  switch (key) {
    F12_THIN_KEYS_2(F12_THIN)
    default: return nullptr;
  }
#undef F12_THIN
}

ThinKernel thin_kernel(int key, bool i5) {
  const int L = ((key >> 6) & 3) + ((key >> 4) & 3) + ((key >> 2) & 3) + (key & 3);
  if (i5) return L <= kThinL5 ? thin_kernel_i5(key) : nullptr;
  if (L <= 2) return thin_kernel_l2(key);
  return L == 3 ? thin_kernel_l3(key) : nullptr;
}

}  // namespace f12k
