// thin_inst.cu -- instances of the thin contraction kernel.  Compiled seven
// times, with F12_THIN_PART = 0..6, each part holding a group of class keys
// (see thin.cuh); part 0 also holds the dispatch over all of them.
#include "thin.cuh"

#ifndef F12_THIN_PART
#error "compile with -DF12_THIN_PART=0..6"
#endif

namespace f12k {

#define F12_CASE_OTHER(K) \
  case K: return i5 ? nullptr : thin_entry<K, false>();
#define F12_CASE_I5(K) \
  case K: return i5 ? thin_entry<K, true>() : nullptr;

#if F12_THIN_PART == 0
ThinKernel thin_part0(int key, bool i5) {
  switch (key) { F12_THIN_KEYS_2(F12_CASE_OTHER) default: return nullptr; }
}

ThinKernel thin_kernel(int key, bool i5) {
  ThinKernel (*const parts[])(int, bool) = {thin_part0, thin_part1, thin_part2, thin_part3,
                                            thin_part4, thin_part5, thin_part6};
  for (auto part : parts)
    if (ThinKernel k = part(key, i5)) return k;
  return nullptr;
}

int thin_slot(int key, bool i5) {
  int i = 0;
#define F12_THIN_IDX(K) \
  if (key == K) return i; \
  ++i;
  F12_THIN_KEYS_2(F12_THIN_IDX)
  if (i5) return -1;
  F12_THIN_KEYS_3(F12_THIN_IDX)
#undef F12_THIN_IDX
  return -1;
}
#elif F12_THIN_PART == 1
ThinKernel thin_part1(int key, bool i5) {
  switch (key) { F12_THIN_KEYS_3A(F12_CASE_OTHER) default: return nullptr; }
}
#elif F12_THIN_PART == 2
ThinKernel thin_part2(int key, bool i5) {
  switch (key) { F12_THIN_KEYS_3B(F12_CASE_OTHER) default: return nullptr; }
}
#elif F12_THIN_PART == 3
ThinKernel thin_part3(int key, bool i5) {
  switch (key) { F12_THIN_KEYS_3C(F12_CASE_OTHER) default: return nullptr; }
}
#elif F12_THIN_PART == 4
ThinKernel thin_part4(int key, bool i5) {
  switch (key) { F12_THIN_KEYS_3D(F12_CASE_OTHER) default: return nullptr; }
}
#elif F12_THIN_PART == 5
ThinKernel thin_part5(int key, bool i5) {
  switch (key) { F12_THIN_KEYS_2A(F12_CASE_I5) default: return nullptr; }
}
#elif F12_THIN_PART == 6
ThinKernel thin_part6(int key, bool i5) {
  switch (key) { F12_THIN_KEYS_2B(F12_CASE_I5) default: return nullptr; }
}
#endif

}  // namespace f12k
