// thin_l2.cu -- instances of the thin contraction for quartets of total order L <= 2 (not I5).
#include "thin.cuh"

namespace f12k {

ThinKernel thin_kernel_l2(int key) {
#define F12_THIN(K) \
  case K: return thin_entry<K, false>();
  switch (key) {
    F12_THIN_KEYS_2(F12_THIN)
    default: return nullptr;
  }
#undef F12_THIN
}

}  // namespace f12k
