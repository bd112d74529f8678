// kernel_common.cuh -- types and helpers shared by the library's kernel
// translation units (f12int.cu: pair data, screening, auxiliary stage,
// general contraction, host API; thin.cu: the thin contraction kernels).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace f12k {

constexpr int kLaux = 14;                          // highest radial order (I5 of f shells)
constexpr int kPartPitch = 16;                     // doubles per family-partial row (128 bytes, whole sectors)
constexpr int kSkipKey = 24 * (kLaux + 1) * 34;    // work-item key of a primitive quartet the screen drops

// Pair data of a basis as the kernels see it (shell-pair tables of Sec. 2.2).
struct PairView {
  const int *pair_start;     // [nshell*nshell + 1] first primitive pair of shell pair (i,j)
  const double *pp_p;        // exponent sum p
  const double *pp_P;        // [6*npp] centre P as heavy centre H (3) + offset P - H (3)
  const double *pp_ab;       // [2*npp] exponents a, b
  const int64_t *pp_eoff;    // offset into epool of this primitive pair's tables
  const double *epool;       // E (3 dims) then F (3 dims), each (la+1)(lb+1)(la+lb+1)
  const int *shell_l;
  int nshell;
  const double *qprim;       // [npp] primitive Schwarz factors of the class, or null
  const double *grow;        // [ngrow] growth G(i kGrowStep) of the class's kernel, or null (no growth)
  int ngrow;
};

// A list of shell quartets.  In a batch (qslot != null) every quartet names a
// slot, which gives the pair data of its basis and the output array of its
// request; counts then live in device memory (count_dev[0] quartets,
// count_dev[1] primitive quartets), so one captured launch sequence serves
// every batch.
struct QuartetView {
  const int32_t *quartets;     // [n][4]
  const int64_t *pq_off;       // [n+1] first primitive quartet of each shell quartet
  int64_t n;
  const int64_t *count_dev;    // batch: {n, pq_off[n]} on the device, else null
  const int32_t *qslot;        // batch: slot of each quartet, else null
  const PairView *slot_view;   // batch: pair data per slot
  double *const *slot_out;     // batch: output array per slot
};


// One block of contraction work: quartet q (index into the list), ket range
// split of nsplit.
struct CTask {
  int32_t q;
  int16_t split, nsplit;
};

__host__ __device__ __forceinline__ int nh_count(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
__host__ __device__ __forceinline__ int ncart(int l) { return (l + 1) * (l + 2) / 2; }
// index of the Hermite triple (t, u, v) in order of t+u+v, then decreasing t, then v
__host__ __device__ __forceinline__ int hidx(int t, int u, int v) {
  int s = t + u + v, w = s - t;
  return s * (s + 1) * (s + 2) / 6 + w * (w + 1) / 2 + v;
}

// X_PQ component k = Q - P = (H_cd - H_ab) + (offset_cd - offset_ab).
__device__ __forceinline__ double pair_sep(const double *ppP, int pab, int pcd, int k) {
  return (ppP[6 * pcd + k] - ppP[6 * pab + k]) + (ppP[6 * pcd + 3 + k] - ppP[6 * pab + 3 + k]);
}

// Thin contraction (thin_*.cu): quartets of total order L <= kThinL (I5:
// L <= kThinL5), one warp per shell quartet, always in FP64 (on the mixed
// path too: there it is faster than the FP32 general kernel).
constexpr int kThinL = 3, kThinL5 = 2;
constexpr int kThinWarps = 4;
using ThinKernel = void (*)(PairView, QuartetView, int, int64_t, const CTask *, int64_t, const int64_t *, const int *,
                            const double *, double *, const int64_t *, unsigned long long *);
// The instance for class key (la << 6 | lb << 4 | lc << 2 | ld), or null.
ThinKernel thin_kernel(int key, bool i5);
// Index of a thin class key among the thin keys of its class kind (the batch
// engine's launch slot), -1 if the key is not thin there.
int thin_slot(int key, bool i5);
constexpr int kThinKeys = 35;   // thin keys of the classes other than I5 (15 for I5)
__host__ __device__ inline bool thin_quartet(int key, int cls) {
  const int L = ((key >> 6) & 3) + ((key >> 4) & 3) + ((key >> 2) & 3) + (key & 3);
  return L <= (cls == 5 ? kThinL5 : kThinL);
}

}  // namespace f12k
