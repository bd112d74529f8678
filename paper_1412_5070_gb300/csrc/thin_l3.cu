// thin_l3.cu -- instances of the thin contraction for quartets of total order L = 3 (not I5).
#include "thin.cuh"

namespace f12k {

ThinKernel thin_kernel_l3(int key) {
#define F12_THIN(K) \
  case K: return thin_entry<K, false>();
  switch (key) {
    F12_THIN_KEYS_3(F12_THIN)
    default: return nullptr;
  }
#undef F12_THIN
}

}  // namespace f12k
