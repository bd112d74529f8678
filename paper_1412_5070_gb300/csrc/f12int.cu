// f12int.cu -- CUDA kernels and C ABI of the F12 integral library (sm_103a).
//
// Stages (arXiv:1412.5070, Sec. 2):
//   1. shell-pair data: p, P, and the Hermite expansion coefficients
//      E_t^{ij} (Eq. AB, Eqs. Erec0-Erect) with their AB derivatives
//      F_t^{ij} = dE_t^{ij}/dAB_x for I5, one thread per primitive pair,
//      resident in device memory for the life of the basis;
//   2. auxiliary functions g_n = D_Q^n B_i per primitive quartet (aux.cuh);
//   3. the Hermite integrals R_tuv = d^t/dQx^t d^u/dQy^u d^v/dQz^v B_i
//      (Eq. ri) by the Cartesian recursion for a radial function
//        R^(n)_{t+1,u,v} = t R^(n+1)_{t-1,u,v} + X_QP R^(n+1)_{t,u,v},
//      which holds because d/dQx D_Q^n B = X_QP D_Q^{n+1} B;
//   4. the contraction of Eq. ii (inner ket sum, then bra sum) and for I5 the
//      combination of Eq. I5byI3_, accumulated over primitive quartets.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/f12int.h"
#include "aux.cuh"
#include "kernel_common.cuh"
#include "auxtab.h"
#include "termlist.h"

using namespace f12dev;
using namespace f12k;

namespace {

constexpr int LSH = 3;                 // highest shell angular momentum
constexpr int NHMAX = 680;             // Hermite indices with t+u+v <= 14
constexpr int BLOCK_CONTRACT = 128;
// ket component order of a contraction task: 100 components at most (f f),
// then the class starts (7 term counts at most for lc + ld <= 6)
constexpr int KORD_CLS = 100;
constexpr int KORD_SIZE = KORD_CLS + 16;
constexpr int BLOCK_AUX = 64;

__constant__ unsigned char c_tuv[NHMAX][3];   // Hermite index -> (t, u, v)
__constant__ unsigned char c_cart[LSH + 3][28][3];  // shell l (<= 5) -> component exponents


// ---------------------------------------------------------------------------
// device status word bits: 1 = an auxiliary series hit its length cap,
// 4 = a quartet needs a radial order above LAUX


// Growth of a kernel with distance, tabulated at this step (screening).
constexpr double kGrowStep = 0.05, kGrowMax = 120.0;
constexpr double kPrimScreen = 1e-26;


// Primitive quartets whose Schwarz product is below kPrimScreen are skipped:
// the skipped contributions stay below the absolute accuracy that elements
// just above 1e-12 need for a relative error of 1e-10.  The diagonal
// integrals behind qprim sample the kernel at short range; a kernel that
// grows with r (Eq. rs12 with B > 0: I2, I3 like e^{Br}, k4 = f f' and
// k6 = f_r f'_r like e^{2Br}) is larger at the separation R = |P - Q| of the
// two charge distributions, whose overlap e^{-xi w^2} reaches out to R + w.
// A candidate is weighed, as the shell screen weighs a shell quartet, by
//   Gamma = max over w = 0, 0.5, .., 3 (units of 1/sqrt(xi)) of G(R + w) e^{-xi w^2}
// (e^{-xi w^2} = e^{-k^2/4} at the k-th sample).
__device__ __forceinline__ bool prim_negligible(const PairView &PV, int pab, int pcd) {
  if (!PV.qprim) return false;
  const double v = PV.qprim[pab] * PV.qprim[pcd];
  if (v >= kPrimScreen) return false;
  if (!PV.grow) return true;
  const double X = pair_sep(PV.pp_P, pab, pcd, 0), Y = pair_sep(PV.pp_P, pab, pcd, 1),
               Z = pair_sep(PV.pp_P, pab, pcd, 2);
  const double p = PV.pp_p[pab], q = PV.pp_p[pcd];
  const double R = sqrt(X * X + Y * Y + Z * Z), hw = 0.5 * sqrt((p + q) / (p * q));
  constexpr double kOverlap[7] = {1.0, 0.77880078307140487, 0.36787944117144233, 0.10539922456186433,
                                  0.018315638888734179, 0.0019304541362277093, 0.00012340980408667956};
  double gam = 0.0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const int i = min(PV.ngrow - 1, (int)((R + k * hw) * (1.0 / kGrowStep)) + 1);
    gam = fmax(gam, PV.grow[i] * kOverlap[k]);
  }
  return v * gam < kPrimScreen;
}

// ------------------------------------------------------------ pair builder --
// E_0^{00} = exp(-(ab/p) X_AB^2)  (Eq. Erec0); upward in i and j with
//   E_t^{i+1,j} = E_{t-1}^{ij}/(2p) + X_PA E_t^{ij} + (t+1) E_{t+1}^{ij}
//   E_t^{i,j+1} = E_{t-1}^{ij}/(2p) + X_PB E_t^{ij} + (t+1) E_{t+1}^{ij}
// (the standard McMurchie-Davidson form equivalent to Eqs. Ereci-Erect, whose
// printed j-recursion carries a stray factor).  F = dE/dAB_x follows by
// differentiating every step: dX_PA/dAB = -b/p, dX_PB/dAB = a/p,
// dE_0^{00}/dAB = -(2ab/p) X_AB E_0^{00}.
__global__ void k_build_pairs(int npp, const int *pp_shell_a, const int *pp_shell_b, const int *pp_prim_a,
                              const int *pp_prim_b, const double *centers, const int *shell_l,
                              const double *exps, const double *coefs, double *pp_p, double *pp_P,
                              double *pp_ab, const int64_t *pp_eoff, double *epool) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npp) return;
  int sa = pp_shell_a[i], sb = pp_shell_b[i];
  int la = shell_l[sa], lb = shell_l[sb];
  double a = exps[pp_prim_a[i]], b = exps[pp_prim_b[i]];
  double da = coefs[pp_prim_a[i]], db = coefs[pp_prim_b[i]];
  double p = a + b;
  pp_p[i] = p;
  pp_ab[2 * i] = a;
  pp_ab[2 * i + 1] = b;
  const int nt = la + lb + 1;
  const int n1 = (la + 1) * (lb + 1) * nt;
  double *E = epool + pp_eoff[i];
  double *F = E + 3 * n1;
  // P is kept as the centre of the larger exponent H plus the offset P - H,
  // and X_PA, X_PB come from X_AB: both stay exact (zero) for one-centre
  // pairs, and X_PQ formed from them keeps its relative accuracy when P and
  // Q nearly coincide; the parity cancellations of one-centre blocks rely on
  // that.
  const bool heavy_a = a >= b;
  for (int k = 0; k < 3; ++k) {
    double A = centers[3 * sa + k], B = centers[3 * sb + k];
    double XAB = A - B, XPA = -(b / p) * XAB, XPB = (a / p) * XAB;
    pp_P[6 * i + k] = heavy_a ? A : B;
    pp_P[6 * i + 3 + k] = heavy_a ? XPA : XPB;
    double K = exp(-a * b / p * XAB * XAB);
    double scale = (k == 0) ? da * db : 1.0;
    double *Ek = E + k * n1, *Fk = F + k * n1;
    for (int j = 0; j < n1; ++j) Ek[j] = Fk[j] = 0.0;
#define EI(ii, jj, t) Ek[((ii) * (lb + 1) + (jj)) * nt + (t)]
#define FI(ii, jj, t) Fk[((ii) * (lb + 1) + (jj)) * nt + (t)]
    EI(0, 0, 0) = K;
    FI(0, 0, 0) = -2.0 * a * b / p * XAB * K;
    const double h = 0.5 / p;
    for (int ii = 0; ii <= la; ++ii) {
      if (ii > 0) {
        for (int t = 0; t <= ii; ++t) {
          double e = XPA * EI(ii - 1, 0, t), f = XPA * FI(ii - 1, 0, t) - b / p * EI(ii - 1, 0, t);
          if (t > 0) {
            e += h * EI(ii - 1, 0, t - 1);
            f += h * FI(ii - 1, 0, t - 1);
          }
          if (t + 1 <= ii - 1) {
            e += (t + 1) * EI(ii - 1, 0, t + 1);
            f += (t + 1) * FI(ii - 1, 0, t + 1);
          }
          EI(ii, 0, t) = e;
          FI(ii, 0, t) = f;
        }
      }
      for (int jj = 1; jj <= lb; ++jj) {
        for (int t = 0; t <= ii + jj; ++t) {
          double e = XPB * EI(ii, jj - 1, t), f = XPB * FI(ii, jj - 1, t) + a / p * EI(ii, jj - 1, t);
          if (t > 0) {
            e += h * EI(ii, jj - 1, t - 1);
            f += h * FI(ii, jj - 1, t - 1);
          }
          if (t + 1 <= ii + jj - 1) {
            e += (t + 1) * EI(ii, jj - 1, t + 1);
            f += (t + 1) * FI(ii, jj - 1, t + 1);
          }
          EI(ii, jj, t) = e;
          FI(ii, jj, t) = f;
        }
      }
    }
#undef EI
#undef FI
    for (int j = 0; j < n1; ++j) {
      Ek[j] *= scale;
      Fk[j] *= scale;
    }
  }
}

// ------------------------------------------------------------------- aux --
__device__ __forceinline__ int64_t qv_count(const QuartetView &QV) { return QV.count_dev ? QV.count_dev[0] : QV.n; }

// Pair data of quartet q: the kernel's own view, or the slot's in a batch
// (a compile-time choice, so that the single-basis kernels keep their view in
// the parameter space).
template <bool BATCH>
__device__ __forceinline__ const PairView &qv_view(const PairView &PV, const QuartetView &QV, int64_t q) {
  if constexpr (BATCH) return QV.slot_view[QV.qslot[q]];
  else return PV;
}


__device__ __forceinline__ int64_t find_quartet(const int64_t *off, int64_t n, int64_t pq) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= pq) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Work items of the auxiliary stage: item = (primitive quartet of the chunk) * nf + family.
struct ItemGeom {
  double xi, D;
  int L;
  int iab, icd;
  const PairView *pv;
};

template <bool BATCH>
__device__ __forceinline__ ItemGeom item_geometry(const PairView &PV0, const QuartetView &QV, int cls, int64_t pq) {
  int64_t q = find_quartet(QV.pq_off, qv_count(QV), pq);
  const PairView &PV = qv_view<BATCH>(PV0, QV, q);
  const int32_t *s = QV.quartets + 4 * q;
  const int ns = PV.nshell;
  int ab = s[0] * ns + s[1], cd = s[2] * ns + s[3];
  int npcd = PV.pair_start[cd + 1] - PV.pair_start[cd];
  int64_t r = pq - QV.pq_off[q];
  int iab = PV.pair_start[ab] + (int)(r / npcd);
  int icd = PV.pair_start[cd] + (int)(r % npcd);
  ItemGeom g;
  g.iab = iab;
  g.icd = icd;
  g.pv = &PV;
  g.L = PV.shell_l[s[0]] + PV.shell_l[s[1]] + PV.shell_l[s[2]] + PV.shell_l[s[3]] + (cls == 5 ? 2 : 0);
  double p = PV.pp_p[iab], qq = PV.pp_p[icd];
  double X = pair_sep(PV.pp_P, iab, icd, 0), Y = pair_sep(PV.pp_P, iab, icd, 1), Z = pair_sep(PV.pp_P, iab, icd, 2);
  g.D = sqrt(X * X + Y * Y + Z * Z);
  g.xi = p * qq / (p + qq);
  return g;
}

__device__ __forceinline__ int item_key(int f, int L, int bin) { return (f * (LAUX + 1) + L) * NZBIN + bin; }
constexpr int SKIP_KEY = kSkipKey;   // last key: negligible primitive quartets
static_assert(kSkipKey == MAXFAM * (LAUX + 1) * NZBIN, "the skip key follows the item keys");
static_assert(kLaux == LAUX, "one highest radial order");

// Pass 1: key of every item and a histogram of the keys.
// Items of a list: (pq_off[n] - pq0) * nf, from the device counts in a batch.
__device__ __forceinline__ int64_t item_count(const QuartetView &QV, int nf, int64_t pq0, int64_t nitems) {
  return QV.count_dev ? (QV.count_dev[1] - pq0) * nf : nitems;
}

// hist[key] += 1 for every active lane, one atomic per distinct key of the warp
__device__ __forceinline__ void hist_add(unsigned int *hist, int key) {
  const unsigned grp = __match_any_sync(__activemask(), key);
  if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&hist[key], (unsigned)__popc(grp));
}

// Pass 1: key of every item and a histogram of the keys.  One thread per
// primitive quartet (its geometry serves all of its families).
template <bool BATCH>
__global__ void k_items_classify(Tables T, PairView PV, QuartetView QV, int cls, int64_t pq0, int64_t nitems,
                                 int *keys, unsigned int *hist) {
  const int kcls = cls == 5 ? 3 : cls;
  const int nf = T.nfam[kcls];
  if (nf <= 0) return;   // a class the factor leaves out (never scheduled)
  const int64_t npq = item_count(QV, nf, pq0, nitems) / nf;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < npq;
       r += (int64_t)gridDim.x * blockDim.x) {
    ItemGeom g = item_geometry<BATCH>(PV, QV, cls, pq0 + r);
    const bool skip = prim_negligible(*g.pv, g.iab, g.icd);
    for (int f = 0; f < nf; ++f) {
      const FamDev &F = T.fam[T.fam0[kcls] + f];
      const int key = skip ? SKIP_KEY : item_key(f, min(g.L, LAUX), item_bin(F, g.xi, g.D, g.L));
      keys[r * nf + f] = key;
      hist_add(hist, key);
    }
  }
}

// Pass 2: exclusive scan of the histogram (one block).
__global__ void k_items_scan(unsigned int *hist, int nkeys) {
  __shared__ unsigned int part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int per = (nkeys + nt - 1) / nt;
  unsigned int s = 0;
  for (int i = tid * per; i < min(nkeys, (tid + 1) * per); ++i) s += hist[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    unsigned int run = 0;
    for (int i = 0; i < nt; ++i) {
      unsigned int v = part[i];
      part[i] = run;
      run += v;
    }
  }
  __syncthreads();
  unsigned int run = part[tid];
  for (int i = tid * per; i < min(nkeys, (tid + 1) * per); ++i) {
    unsigned int v = hist[i];
    hist[i] = run;
    run += v;
  }
}

// Pass 3: scatter item indices into key order (order inside a key is free:
// every item is evaluated independently, so results do not depend on it).
__global__ void k_items_scatter(QuartetView QV, int nf, int64_t pq0, const int *keys, unsigned int *cursor,
                                int64_t nitems, unsigned int *order) {
  const int64_t nit = item_count(QV, nf, pq0, nitems);
  const int lane = threadIdx.x & 31;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nit;
       it += (int64_t)gridDim.x * blockDim.x) {
    // one atomic per distinct key of the warp; lanes take consecutive slots
    const int key = keys[it];
    const unsigned grp = __match_any_sync(__activemask(), key);
    const int leader = __ffs(grp) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&cursor[key], (unsigned)__popc(grp));
    base = __shfl_sync(grp, base, leader);
    order[base + __popc(grp & ((1u << lane) - 1u))] = (unsigned int)it;
  }
}

// Pass 4: one family's contribution to hat g_l (l <= L) per item, into
// part[item * kPartPitch + l], in key order; the row is written up to the end
// of the 32-byte sector that holds order L (zeros past L), so that no sector
// is left partly written.  The families evaluated by
// quadrature (b < 0 or a lowest power below -1, FamDev::quad) are left to a
// second launch of the same kernel with QUAD = true (family_quad), made only
// when the factor has such families.
template <bool BATCH, bool QUAD>
__device__ __forceinline__ unsigned long long items_eval_one(Tables T, PairView PV, QuartetView QV, int cls,
                                                             int64_t pq0, int64_t it, const int *keys, double *part,
                                                             unsigned int *status) {
  // a primitive quartet the screen dropped (decided once, by the classify
  // pass) is never read by the contraction
  if (keys[it] == SKIP_KEY) return 0;
  const int kcls = cls == 5 ? 3 : cls;
  const int nf = T.nfam[kcls];
  const int64_t pq = pq0 + it / nf;
  const int f = (int)(it % nf);
  const FamDev &F = T.fam[T.fam0[kcls] + f];
  if ((F.quad != 0) != QUAD) return 0;   // the other launch's family
  ItemGeom g = item_geometry<BATCH>(PV, QV, cls, pq);
  if (g.L > LAUX) {
    atomicOr(status, 4u);
    return 0;
  }
  double out[LAUX + 1];
  for (int l = 0; l <= g.L; ++l) out[l] = 0.0;
  unsigned long long nfma = 0;
  int bad = family_eval<QUAD>(T, F, g.xi, g.D, g.L, out, &nfma);
  if (bad) atomicOr(status, 1u);
  double2 *o = reinterpret_cast<double2 *>(part + it * kPartPitch);
  for (int l = 0; l <= (g.L | 3); l += 2)
    o[l >> 1] = make_double2(l <= g.L ? out[l] : 0.0, l + 1 <= g.L ? out[l + 1] : 0.0);
  return nfma;
}

template <bool BATCH, bool QUAD = false>
__global__ void k_items_eval(Tables T, PairView PV, QuartetView QV, int cls, int64_t pq0, int64_t nitems,
                             const unsigned int *order, const int *keys, double *part, unsigned int *status,
                             unsigned long long *fma_total) {
  unsigned long long nfma = 0;
  if constexpr (BATCH) {
    const int64_t nit = item_count(QV, T.nfam[cls == 5 ? 3 : cls], pq0, nitems);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nit; t += (int64_t)gridDim.x * blockDim.x)
      nfma += items_eval_one<BATCH, QUAD>(T, PV, QV, cls, pq0, order[t], keys, part, status);
  } else {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nitems) nfma = items_eval_one<BATCH, QUAD>(T, PV, QV, cls, pq0, order[t], keys, part, status);
  }
  // warp-aggregated count of the core multiply-adds (series terms and quadrature nodes)
  if (fma_total) {
    for (int o = 16; o > 0; o >>= 1) nfma += __shfl_down_sync(0xffffffffu, nfma, o);
    if ((threadIdx.x & 31) == 0 && nfma) atomicAdd(fma_total, nfma);
  }
}



// hat g_n at given (xi, D) points (no prefactor), for the aux-stage tests.
__global__ void k_aux_points(Tables T, int cls, int64_t npts, const double *xi, const double *D, int nmax,
                             double *out, unsigned int *status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npts) return;
  double g[LAUX + 1];
  int bad = aux_eval(T, cls == 5 ? 3 : cls, xi[i], D[i], nmax, g);
  if (bad) atomicOr(status, 1u);
  for (int n = 0; n <= nmax; ++n) out[i * (nmax + 1) + n] = g[n];
}

// -------------------------------------------------------------- contract --
// One block per shell quartet and range of ket components: a quartet whose
// buffers would not fit in shared memory is split into NSPLIT blocks, each
// owning a contiguous range of the c*d Cartesian components (every block
// repeats the Hermite recursion, which is a small part of the work at the
// angular momenta that need a split).  The NW warps of a block split the ket
// primitive pairs.  Below, ncd is the number of ket components of the block.
// Shared memory (doubles):
//   per warp: R0, R1  two levels of the Hermite recursion        2 * nh(L)
//             Rc      the last level (n = 0) in a cube [t][u][v] of
//                     pitch L+1, so that the index of R_{t+t',u+u',v+v'}
//                     is a bra part plus a ket part                  (L+1)^3
//             W       ket-contracted integrals, bra order <= lab
//                     (+2 for I5), summed over the warp's ket
//                     primitive pairs                             nh(Lb) * ncd
//             g       the radial derivatives g_n                  LAUX + 1
//             E3cd    E^{cd}_{t'u'v'} = E_t' E_u' E_v' of the
//                     current ket primitive pair, per component   ne3(lc, ld)
//   block:    O       output accumulator                          nab * ncd
//             ck, hb  (ints) cube offset of every ket Hermite product
//                     and W offset hidx(t,u,v)*ncd of every bra one
//             E3ab    E^{ab}_{tuv} of the current bra primitive
//                     pair (times (a-b)/2p for I5), and for I5 the
//                     three dE/dAB-weighted products              ne3(la, lb) (x4 for I5)
// The per-warp W are summed in warp order, so results do not depend on
// scheduling; the sum also applies the bra sign (-1)^{t+u+v} of Eq. ii.
__host__ __device__ __forceinline__ size_t contract_warp_doubles(int nhL, int nhB, int ncd, int ne3cd, int L) {
  return (size_t)2 * nhL + (size_t)(L + 1) * (L + 1) * (L + 1) + (size_t)nhB * ncd + (LAUX + 1) + (size_t)ne3cd;
}

// number of Hermite products over all component pairs of shells (l1, l2)
__host__ __device__ inline int ne3_count(int l1, int l2) {
  int n = 0;
  for (int i = l1; i >= 0; --i)
    for (int j = l1 - i; j >= 0; --j)
      for (int i2 = l2; i2 >= 0; --i2)
        for (int j2 = l2 - i2; j2 >= 0; --j2) n += (i + i2 + 1) * (j + j2 + 1) * (l1 - i - j + l2 - i2 - j2 + 1);
  return n;
}

// largest number of Hermite products over the ranges of jc consecutive
// component pairs (same lexicographic order as the kernel's)
static inline int ne3_chunk_max(int l1, int l2, int jc) {
  int best = 0, cur = 0, k = 0;
  for (int i = l1; i >= 0; --i)
    for (int j = l1 - i; j >= 0; --j)
      for (int i2 = l2; i2 >= 0; --i2)
        for (int j2 = l2 - i2; j2 >= 0; --j2) {
          cur += (i + i2 + 1) * (j + j2 + 1) * (l1 - i - j + l2 - i2 - j2 + 1);
          if (++k == jc) {
            best = cur > best ? cur : best;
            cur = k = 0;
          }
        }
  return cur > best ? cur : best;
}

__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }

// One contraction task (quartet and ket range) by the whole block.  T is the
// type of the Hermite recursion, the E products and every accumulation
// (double, or float on the mixed path); g_n are always summed in double.
template <bool BATCH, class T>
__device__ __forceinline__ void contract_task(const PairView &PV0, const QuartetView &QV, int cls, int nf,
                                              int64_t pq0, const CTask task, const int *keys, const double *part,
                                              double *out,
                                              const int64_t *offsets, unsigned long long *flops_total,
                                              T *smem, int *off_ab, int *off_cd, int *kord) {
  const int64_t q = task.q;
  const int split = task.split, nsplit = task.nsplit;
  const PairView &PV = qv_view<BATCH>(PV0, QV, q);
  const int32_t *s = QV.quartets + 4 * q;
  const int ns = PV.nshell;
  const int la = PV.shell_l[s[0]], lb = PV.shell_l[s[1]], lc = PV.shell_l[s[2]], ld = PV.shell_l[s[3]];
  const int ext = cls == 5 ? 2 : 0;
  const int lab = la + lb, lcd = lc + ld;
  const int L = lab + lcd + ext;
  const int Lb = lab + ext;
  const int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
  const int ncd_all = nc * nd, nab = na * nb;
  const int jc = (ncd_all + nsplit - 1) / nsplit, j0 = split * jc;
  const int ncd = min(jc, ncd_all - j0);   // ket components of this block: j0 .. j0+ncd-1
  if (ncd <= 0) return;                     // block-uniform
  const int nhL = nh_count(L), nhB = nh_count(Lb);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  if (tid == 0) {
    int o = 0;
    for (int j = 0; j < ncd; ++j) {
      off_cd[j] = o;
      const unsigned char *ec = c_cart[lc][(j0 + j) / nd], *ed = c_cart[ld][(j0 + j) % nd];
      o += (ec[0] + ed[0] + 1) * (ec[1] + ed[1] + 1) * (ec[2] + ed[2] + 1);
    }
    off_cd[ncd] = o;
    // ket components in order of increasing term count (the ket step's loop
    // length), one class per count: kord[0..ncd) the components,
    // kord[KORD_CLS + c] the first position of class c (ncd after the last).
    // Lanes that take consecutive entries of the (class, bra index,
    // component) order run loops of one length.
    int nc_ = 0, pos = 0;
    while (pos < ncd) {
      int len = 1 << 30;
      for (int j = 0; j < ncd; ++j) {
        const int lj = off_cd[j + 1] - off_cd[j];
        if (lj > (nc_ ? off_cd[kord[pos - 1] + 1] - off_cd[kord[pos - 1]] : 0) && lj < len) len = lj;
      }
      kord[KORD_CLS + nc_] = pos;
      for (int j = 0; j < ncd; ++j)
        if (off_cd[j + 1] - off_cd[j] == len) kord[pos++] = j;
      ++nc_;
    }
    kord[KORD_CLS + nc_] = ncd;
    o = 0;
    for (int j = 0; j < nab; ++j) {
      off_ab[j] = o;
      const unsigned char *ea = c_cart[la][j / nb], *eb = c_cart[lb][j % nb];
      o += (ea[0] + eb[0] + 1) * (ea[1] + eb[1] + 1) * (ea[2] + eb[2] + 1);
    }
    off_ab[nab] = o;
  }
  __syncthreads();
  const int ne3cd = off_cd[ncd], ne3ab = off_ab[nab];
  const size_t wsz = contract_warp_doubles(nhL, nhB, ncd, ne3cd, L);
  const int P = L + 1;   // cube pitch of Rc
  T *R0 = smem + warp * wsz;
  T *R1 = R0 + nhL;
  T *Rc = R1 + nhL;
  T *W = Rc + (size_t)P * P * P;
  T *gw = W + (size_t)nhB * ncd;
  T *E3cd = gw + (LAUX + 1);
  T *Oacc = smem + nw * wsz;
  T *E3ab = Oacc + (size_t)nab * ncd;
  T *E3fx = E3ab + ne3ab, *E3fy = E3fx + ne3ab, *E3fz = E3fy + ne3ab;
  int *ck = reinterpret_cast<int *>(E3ab + (size_t)ne3ab * (cls == 5 ? 4 : 1));
  int *hb = ck + ne3cd;
  // index tables of this task (same for every primitive quartet)
  for (int j = tid; j < ncd; j += nthr) {
    const unsigned char *ec = c_cart[lc][(j0 + j) / nd], *ed = c_cart[ld][(j0 + j) % nd];
    const int tx = ec[0] + ed[0], ty = ec[1] + ed[1], tz = ec[2] + ed[2];
    int m = off_cd[j];
    for (int t2 = 0; t2 <= tx; ++t2)
      for (int u2 = 0; u2 <= ty; ++u2)
        for (int v2 = 0; v2 <= tz; ++v2) ck[m++] = (t2 * P + u2) * P + v2;
  }
  for (int c = tid; c < nab; c += nthr) {
    const unsigned char *ea = c_cart[la][c / nb], *eb = c_cart[lb][c % nb];
    const int tx = ea[0] + eb[0], ty = ea[1] + eb[1], tz = ea[2] + eb[2];
    int m = off_ab[c];
    for (int t = 0; t <= tx; ++t)
      for (int u = 0; u <= ty; ++u)
        for (int v = 0; v <= tz; ++v) hb[m++] = hidx(t, u, v) * ncd;
  }
  __syncthreads();
  const int ab = s[0] * ns + s[1], cd = s[2] * ns + s[3];
  const int ab0 = PV.pair_start[ab], npab = PV.pair_start[ab + 1] - ab0;
  const int cd0 = PV.pair_start[cd], npcd = PV.pair_start[cd + 1] - cd0;
  const int ntab = lab + 1, ntcd = lcd + 1;
  const int n1ab = (la + 1) * (lb + 1) * ntab;
  const int n1cd = (lc + 1) * (ld + 1) * ntcd;
  const double pi52 = 17.493418327624862846;  // pi^{5/2}

  for (int i = tid; i < nab * ncd; i += nthr) Oacc[i] = 0.0;
  unsigned long long nproc = 0;   // primitive quartets this warp processed

  for (int iab = 0; iab < npab; ++iab) {
    const int pab = ab0 + iab;
    for (int i = lane; i < nhB * ncd; i += 32) W[i] = 0.0;
    __syncwarp();
    for (int icd = warp; icd < npcd; icd += nw) {
      const int pcd = cd0 + icd;
      const int64_t pq = QV.pq_off[q] + (int64_t)iab * npcd + icd - pq0;
      if (keys[pq * nf] == SKIP_KEY) continue;   // dropped by the primitive screen; warp-uniform
      ++nproc;
      const T X = (T)pair_sep(PV.pp_P, pab, pcd, 0), Y = (T)pair_sep(PV.pp_P, pab, pcd, 1),
                   Z = (T)pair_sep(PV.pp_P, pab, pcd, 2);
      // g_n = sqrt(pi^5/(p+q))/(pq) * sum over families (fixed order)
      if (lane <= L) {
        const double p = PV.pp_p[pab], qq = PV.pp_p[pcd];
        double acc = 0.0;
        for (int fm = 0; fm < nf; ++fm) acc += part[(pq * nf + fm) * kPartPitch + lane];
        gw[lane] = (T)(pi52 / (sqrt(p + qq) * p * qq) * acc);
      }
      // E^{cd}_{t'u'v'} products of this ket primitive pair
      const double *Ecd = PV.epool + PV.pp_eoff[pcd];
      for (int j = lane; j < ncd; j += 32) {
        const unsigned char *ec = c_cart[lc][(j0 + j) / nd], *ed = c_cart[ld][(j0 + j) % nd];
        const double *ex = Ecd + (ec[0] * (ld + 1) + ed[0]) * ntcd;
        const double *ey = Ecd + n1cd + (ec[1] * (ld + 1) + ed[1]) * ntcd;
        const double *ez = Ecd + 2 * n1cd + (ec[2] * (ld + 1) + ed[2]) * ntcd;
        const int tx = ec[0] + ed[0], ty = ec[1] + ed[1], tz = ec[2] + ed[2];
        T *e = E3cd + off_cd[j];
        int m = 0;
        for (int t2 = 0; t2 <= tx; ++t2)
          for (int u2 = 0; u2 <= ty; ++u2) {
            const double exy = ex[t2] * ey[u2];
            for (int v2 = 0; v2 <= tz; ++v2) e[m++] = (T)(exy * ez[v2]);
          }
      }
      __syncwarp();
      // Hermite recursion from level n = L down to 0, ping-pong between R0/R1
      T *cur = R0, *nxt = R1;
      if (lane == 0) {
        cur[0] = gw[L];
        if (L == 0) Rc[0] = gw[0];
      }
      __syncwarp();
      for (int n = L - 1; n >= 0; --n) {
        const int cnt = nh_count(L - n);
        for (int idx = lane; idx < cnt; idx += 32) {
          const int t = c_tuv[idx][0], u = c_tuv[idx][1], v = c_tuv[idx][2];
          T val;
          if (idx == 0) {
            val = gw[n];
          } else if (t > 0) {
            val = X * cur[hidx(t - 1, u, v)];
            if (t > 1) val += (t - 1) * cur[hidx(t - 2, u, v)];
          } else if (u > 0) {
            val = Y * cur[hidx(t, u - 1, v)];
            if (u > 1) val += (u - 1) * cur[hidx(t, u - 2, v)];
          } else {
            val = Z * cur[hidx(t, u, v - 1)];
            if (v > 1) val += (v - 1) * cur[hidx(t, u, v - 2)];
          }
          if (n > 0) nxt[idx] = val;
          else Rc[(t * P + u) * P + v] = val;   // the last level, in the cube
        }
        __syncwarp();
        T *tmp = cur;
        cur = nxt;
        nxt = tmp;
      }
      // inner (ket) sum of Eq. ii:  W[tuv][cd] += sum E^{cd}_{t'u'v'} R_{t+t',u+u',v+v'},
      // entries taken in (term-count class, bra index, component) order
      for (int r = lane, c = 0; r < nhB * ncd; r += 32) {
        while (r >= nhB * kord[KORD_CLS + c + 1]) ++c;
        const int c0 = kord[KORD_CLS + c], n_c = kord[KORD_CLS + c + 1] - c0;
        const int rr = r - nhB * c0;
        const int bi = rr / n_c;
        const int j = kord[c0 + rr - bi * n_c];
        const int cb = (c_tuv[bi][0] * P + c_tuv[bi][1]) * P + c_tuv[bi][2];
        const int m0 = off_cd[j], m1 = off_cd[j + 1];
        T acc = 0;
        for (int m = m0; m < m1; ++m) acc = tfma(E3cd[m], Rc[cb + ck[m]], acc);
        W[bi * ncd + j] += acc;
      }
      __syncwarp();
    }
    __syncthreads();
    // sum the warps' W into warp 0's buffer (fixed order), with the bra sign
    const size_t woff = (size_t)2 * nhL + (size_t)P * P * P;   // W within a warp's region
    T *W0 = smem + woff;
    for (int i = tid; i < nhB * ncd; i += nthr) {
      T acc = W0[i];
      for (int w = 1; w < nw; ++w) acc += smem[w * wsz + woff + i];
      const int bi = i / ncd;
      W0[i] = ((c_tuv[bi][0] + c_tuv[bi][1] + c_tuv[bi][2]) & 1) ? -acc : acc;
    }
    // E^{ab}_{tuv} products of this bra primitive pair
    const double *Eab = PV.epool + PV.pp_eoff[pab];
    const double *Fab = Eab + 3 * n1ab;
    const double a = PV.pp_ab[2 * pab], b = PV.pp_ab[2 * pab + 1];
    const double c5 = (a - b) / (2.0 * (a + b));
    for (int c = tid; c < nab; c += nthr) {
      const unsigned char *ea = c_cart[la][c / nb], *eb = c_cart[lb][c % nb];
      const int ox = (ea[0] * (lb + 1) + eb[0]) * ntab;
      const int oy = n1ab + (ea[1] * (lb + 1) + eb[1]) * ntab;
      const int oz = 2 * n1ab + (ea[2] * (lb + 1) + eb[2]) * ntab;
      const int tx = ea[0] + eb[0], ty = ea[1] + eb[1], tz = ea[2] + eb[2];
      const int o = off_ab[c];
      int m = 0;
      for (int t = 0; t <= tx; ++t)
        for (int u = 0; u <= ty; ++u)
          for (int v = 0; v <= tz; ++v, ++m) {
            const double exy = Eab[ox + t] * Eab[oy + u];
            if (cls != 5) {
              E3ab[o + m] = (T)(exy * Eab[oz + v]);
            } else {
              E3ab[o + m] = (T)(c5 * exy * Eab[oz + v]);
              E3fx[o + m] = (T)(Fab[ox + t] * Eab[oy + u] * Eab[oz + v]);
              E3fy[o + m] = (T)(Eab[ox + t] * Fab[oy + u] * Eab[oz + v]);
              E3fz[o + m] = (T)(exy * Fab[oz + v]);
            }
          }
    }
    __syncthreads();
    // outer (bra) sum
    for (int i = tid; i < nab * ncd; i += nthr) {
      const int iabc = i / ncd, j = i - iabc * ncd;
      const int ia = iabc / nb, ib = iabc - ia * nb;
      const unsigned char *ea = c_cart[la][ia], *eb = c_cart[lb][ib];
      const int tx = ea[0] + eb[0], ty = ea[1] + eb[1], tz = ea[2] + eb[2];
      const int o = off_ab[iabc];
      T acc = 0;
      int m = 0;
      for (int t = 0; t <= tx; ++t)
        for (int u = 0; u <= ty; ++u)
          for (int v = 0; v <= tz; ++v, ++m) {
            if (cls != 5) {
              acc = tfma(E3ab[o + m], W0[hb[o + m] + j], acc);
            } else {
              // Eq. I5byI3_ with the second coefficient -1 (see the derivation note
              // below); W0 carries the bra sign, so the gradient term changes sign
              const T lap = W0[hidx(t + 2, u, v) * ncd + j] + W0[hidx(t, u + 2, v) * ncd + j] +
                                 W0[hidx(t, u, v + 2) * ncd + j];
              acc = tfma(E3ab[o + m], lap, acc);
              acc = tfma(E3fx[o + m], W0[hidx(t + 1, u, v) * ncd + j], acc);
              acc = tfma(E3fy[o + m], W0[hidx(t, u + 1, v) * ncd + j], acc);
              acc = tfma(E3fz[o + m], W0[hidx(t, u, v + 1) * ncd + j], acc);
            }
          }
      Oacc[i] += acc;
    }
    __syncthreads();
  }
  double *o;
  if constexpr (BATCH) o = QV.slot_out[QV.qslot[q]] + offsets[q];
  else o = out + offsets[q];
  for (int i = tid; i < nab * ncd; i += nthr) {
    const int iabc = i / ncd;
    o[(size_t)iabc * ncd_all + j0 + (i - iabc * ncd)] = (double)Oacc[i];
  }
  if (flops_total && lane == 0 && nproc) {
    // algorithmic FP64 flops per primitive quartet: Hermite recursion 2 C(L+4,4)
    // (counted once per quartet, not per split), ket step 2 nh(lab+ext) nh(lcd)
    // ncd, bra step 2 nab nh(lab) ncd (x4 for I5)
    const unsigned long long r = split == 0 ? 2ull * (L + 1) * (L + 2) * (L + 3) * (L + 4) / 24 : 0ull;
    const unsigned long long ket = 2ull * nhB * nh_count(lcd) * ncd;
    const unsigned long long bra = 2ull * nab * nh_count(lab) * ncd * (cls == 5 ? 4 : 1);
    atomicAdd(flops_total, nproc * (r + ket + bra));
  }
}

template <bool BATCH, class T>
__global__ void __launch_bounds__(BLOCK_CONTRACT)
k_contract(PairView PV0, QuartetView QV, int cls, int nf, int64_t pq0, const CTask *tasks, int64_t ntask,
           const int64_t *ntask_dev, const int *keys, const double *part, double *out, const int64_t *offsets,
           unsigned int *status, unsigned long long *flops_total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smem = reinterpret_cast<T *>(smem_raw);
  __shared__ int off_ab[101], off_cd[101], kord[KORD_SIZE];
  if constexpr (BATCH) {
    // ntask_dev = {first, end} of this launch's tasks
    const int64_t te = ntask_dev[1];
    for (int64_t tk = ntask_dev[0] + blockIdx.x; tk < te; tk += gridDim.x) {
      __syncthreads();   // the previous task's shared-memory reads are done
      contract_task<BATCH, T>(PV0, QV, cls, nf, pq0, tasks[tk], keys, part, out, offsets, flops_total, smem, off_ab,
                              off_cd, kord);
    }
  } else {
    if (blockIdx.x < ntask)
      contract_task<BATCH, T>(PV0, QV, cls, nf, pq0, tasks[blockIdx.x], keys, part, out, offsets, flops_total, smem,
                              off_ab, off_cd, kord);
  }
}
// Derivation note for I5: with d/dA_x = (a/p) d/dP_x + d/dAB_x and
// d/dB_x = (b/p) d/dP_x - d/dAB_x (E depends on AB only, R on P only),
//   1/2 (lap_A - lap_B) = sum_x [ (a-b)/(2p) d^2/dP_x^2 + d/dP_x d/dAB_x ],
// and d/dP_x = -d/dQ_x on R; hence the coefficient of the gradient term is
// -(a+b)/p = -1.

}  // namespace

// ================================================================ host API ==

namespace {
struct Engine;   // batched requests (engine.cuh)
}

struct f12int_ctx {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;
  cudaStream_t stream = nullptr;
  int64_t launches = 0;
  unsigned int *d_status = nullptr;
  // factor tables
  bool factor_ready = false;
  FamDev *d_fam = nullptr;
  double *d_coef = nullptr;
  GroupDev *d_grp = nullptr;
  size_t grp_bytes = 0;
  double *d_jtab = nullptr;   // start-value tables of the series families
  size_t jtab_bytes = 0;
  Tables tables{};
  size_t fam_bytes = 0, coef_bytes = 0;
  // basis
  struct BasisData {
    int nshell = 0;
    int *d_shell_l = nullptr;
    double *d_centers = nullptr;
    int *d_pair_start = nullptr;
    double *d_pp_p = nullptr, *d_pp_P = nullptr, *d_pp_ab = nullptr, *d_epool = nullptr;
    int64_t *d_pp_eoff = nullptr;
    std::vector<int> l, nprim, pair_start;
    std::vector<double> centers, exps, coefs;
    size_t bytes = 0;
    bool prim_screen = true;            // false for the internal per-primitive basis
    double *d_qprim[7] = {nullptr};     // primitive Schwarz factors per class (lazily built)
    std::vector<double> pair_bound[7];  // shell-pair bounds sqrt(max |(ab|k|ab)|) per class (lazily built)
    std::vector<double> pair_cen;       // [nshell^2][3] centre of the most diffuse primitive pair
    std::vector<double> pair_pmin;      // [nshell^2] its exponent sum
  };
  std::deque<BasisData> bases;   // deque: growing it never moves existing entries
  // scratch of compute_class (grown on demand, bounded by the budget)
  int64_t *d_pqoff = nullptr;
  int *d_keys = nullptr;
  unsigned *d_order = nullptr, *d_hist = nullptr;
  double *d_part = nullptr;
  int32_t *d_qperm = nullptr;
  int64_t *d_operm = nullptr;
  CTask *d_tasks = nullptr;
  size_t pqoff_cap = 0, keys_cap = 0, order_cap = 0, hist_cap = 0, part_cap = 0, qperm_cap = 0, operm_cap = 0;
  size_t tasks_cap = 0;
  // optional per-kernel timing (events on the launching stream) and counters
  bool timing = false;
  unsigned long long *d_fma = nullptr;
  double aux_ms = 0.0, contract_ms = 0.0;
  int64_t aux_launches = 0, contract_launches = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_aux, ev_con, ev_pool;
  std::vector<int> h_nw;       // warps per contraction block, per quartet in the working order
  std::vector<int> h_split;    // ket-component ranges (blocks) per quartet, same order
  std::vector<char> h_fp32;    // 1: Hermite recursion and contraction in FP32 (mixed path), same order
  std::vector<size_t> h_smem;  // contraction shared memory, per quartet in the working order
  std::vector<int16_t> h_thin; // class key of a quartet for k_contract_thin, -1: the general kernel; same order
  std::mutex mu;
  std::recursive_mutex bounds_mu;   // first-time primitive and shell-pair bounds
  bool cls_ok[7] = {false, false, false, false, false, false, false};   // classes the factor supports
  bool cls_quad[7] = {false, false, false, false, false, false, false};   // classes with quadrature families
  // growth of each class's kernel with distance (screening estimate):
  // kgrow[cls][i] = G(i * kGrowStep), see screen_estimate
  std::vector<double> kgrow[7];
  // the same tables on the device for the primitive screen ([7][kgrow_n]);
  // grows[cls]: the kernel of cls grows (G > 1 somewhere)
  double *d_kgrow = nullptr;
  size_t kgrow_bytes = 0;
  int kgrow_n = 0;
  bool grows[7] = {false, false, false, false, false, false, false};
  int series_cap = KMAX;   // f12int_set_series_cap
  double plan_ms = 0.0;    // host planning of compute_class calls (f12int_host_stats)
  int64_t plan_calls = 0;
  Engine *engine = nullptr;
};

namespace {

int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return F12INT_ENOMEM;
  return F12INT_ECUDA;
}

#define CK(call)                                    \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_);    \
  } while (0)

template <class T>
int dalloc(f12int_ctx *ctx, T **p, size_t bytes) {
  if (bytes == 0) bytes = 8;
  if (ctx->budget && ctx->used + bytes > ctx->budget) return F12INT_ENOMEM;
  cudaError_t e = cudaMalloc((void **)p, bytes);
  if (e != cudaSuccess) return cuda_fail(e);
  ctx->used += bytes;
  return F12INT_OK;
}

template <class T>
void dfree(f12int_ctx *ctx, T *&p, size_t bytes) {
  if (p) {
    cudaFree(p);
    ctx->used -= std::min(ctx->used, bytes ? bytes : (size_t)8);
    p = nullptr;
  }
}

cudaStream_t pick_stream(f12int_ctx *ctx, void *s) { return s ? (cudaStream_t)s : ctx->stream; }

// NVTX range over a host scope (the stages of a call, visible in a profiler's
// timeline; free when no tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// The pair data of a basis as the kernels see it, for class cls: with the
// primitive screen (its Schwarz factors and the kernel's growth table) when
// screen is set and the factors exist.
PairView pair_view(const f12int_ctx *ctx, const f12int_ctx::BasisData &B, int cls, bool screen) {
  PairView v{B.d_pair_start, B.d_pp_p, B.d_pp_P, B.d_pp_ab, B.d_pp_eoff, B.d_epool, B.d_shell_l, B.nshell,
             nullptr, nullptr, 0};
  if (screen && B.d_qprim[cls]) {
    v.qprim = B.d_qprim[cls];
    if (ctx->grows[cls] && ctx->d_kgrow) {
      v.grow = ctx->d_kgrow + (size_t)cls * ctx->kgrow_n;
      v.ngrow = ctx->kgrow_n;
    }
  }
  return v;
}

bool g_const_ready = false;
std::mutex g_const_mu;

int upload_constants() {
  std::lock_guard<std::mutex> lk(g_const_mu);
  if (g_const_ready) return F12INT_OK;
  unsigned char tuv[NHMAX][3];
  for (int s = 0; s <= 14; ++s)
    for (int t = s; t >= 0; --t)
      for (int v = 0; v <= s - t; ++v) {
        int u = s - t - v;
        int i = hidx(t, u, v);
        tuv[i][0] = (unsigned char)t;
        tuv[i][1] = (unsigned char)u;
        tuv[i][2] = (unsigned char)v;
      }
  unsigned char cart[LSH + 3][28][3];
  std::memset(cart, 0, sizeof(cart));
  for (int l = 0; l < LSH + 3; ++l) {
    int k = 0;
    for (int i = l; i >= 0; --i)
      for (int j = l - i; j >= 0; --j) {
        cart[l][k][0] = (unsigned char)i;
        cart[l][k][1] = (unsigned char)j;
        cart[l][k][2] = (unsigned char)(l - i - j);
        ++k;
      }
  }
  static AuxConst ac;
  fill_aux_const(ac);
  CK(cudaMemcpyToSymbol(c_cratio, ac.cratio, sizeof(ac.cratio)));
  CK(cudaMemcpyToSymbol(c_inv_dfact, ac.inv_dfact, sizeof(ac.inv_dfact)));
  CK(cudaMemcpyToSymbol(d_kum_inv, ac.kum_inv, sizeof(ac.kum_inv)));
  CK(cudaMemcpyToSymbol(d_sm1_ratio, ac.sm1_ratio, sizeof(ac.sm1_ratio)));
  CK(cudaMemcpyToSymbol(d_cser, ac.cser, sizeof(ac.cser)));
  CK(cudaMemcpyToSymbol(d_vstep, ac.vstep, sizeof(ac.vstep)));
  CK(cudaMemcpyToSymbol(d_quarter, ac.quarter, sizeof(ac.quarter)));
  {
    // the Kummer table of the b = 0 families (13.5 MB), kept for the process
    std::vector<double> kt;
    fill_kummer_table(kt);
    double *dk = nullptr;
    CK(cudaMalloc(&dk, sizeof(double) * kt.size()));
    CK(cudaMemcpy(dk, kt.data(), sizeof(double) * kt.size(), cudaMemcpyHostToDevice));
    const double *dkc = dk;
    CK(cudaMemcpyToSymbol(d_mtab, &dkc, sizeof(dkc)));
  }
  CK(cudaMemcpyToSymbol(c_tuv, tuv, sizeof(tuv)));
  CK(cudaMemcpyToSymbol(c_cart, cart, sizeof(cart)));
  CK(cudaMemcpyToSymbol(c_gh_x, ac.gh_x, sizeof(ac.gh_x)));
  CK(cudaMemcpyToSymbol(c_gh_w, ac.gh_w, sizeof(ac.gh_w)));
  CK(cudaMemcpyToSymbol(c_gl_x, ac.gl_x, sizeof(ac.gl_x)));
  CK(cudaMemcpyToSymbol(c_gl_w, ac.gl_w, sizeof(ac.gl_w)));
  g_const_ready = true;
  return F12INT_OK;
}

bool finite_factor(const f12int_factor &f) {
  return std::isfinite(f.c0) && std::isfinite(f.rho) && std::isfinite(f.B) && std::isfinite(f.mu);
}

// A factor given as terms: 1..64 finite terms with g >= 0, not all zero.
int check_terms(const f12int_term *t, int n, f12::TermList &out) {
  if (!t || n < 1 || n > 64) return F12INT_EINVAL;
  out.clear();
  for (int i = 0; i < n; ++i) {
    const f12int_term &u = t[i];
    if (!std::isfinite(u.c) || !std::isfinite(u.a) || !std::isfinite(u.b) || !std::isfinite(u.g) || u.g < 0.0)
      return F12INT_EDOMAIN;
    out.push_back({u.c, u.a, u.b, u.g});
  }
  f12::simplify(out);
  return out.empty() ? F12INT_EDOMAIN : F12INT_OK;
}

int check_factor(const f12int_factor &f) {
  if (!finite_factor(f)) return F12INT_EDOMAIN;
  if (!(f.mu > 0.0) || f.c0 < 0.0 || f.n < 0 || f.n > 20) return F12INT_EDOMAIN;
  if (f.c0 > 0.0 && !(f.rho + 2.0 * f.n + 2.0 > 0.0)) return F12INT_EDOMAIN;
  return F12INT_OK;
}

}  // namespace

extern "C" {

static void collect_events(f12int_ctx *ctx);

const char *f12int_strerror(int status) {
  switch (status) {
    case F12INT_OK: return "ok";
    case F12INT_EINVAL: return "invalid argument";
    case F12INT_ENOMEM: return "device memory budget exceeded";
    case F12INT_EDOMAIN: return "correlation-factor parameters outside the supported domain";
    case F12INT_ENOTREADY: return "basis or correlation factor not set";
    case F12INT_ETIMEOUT: return "timed out";
    case F12INT_ECUDA: return "CUDA runtime error";
    case F12INT_EDEVICE: return "device-side check failed";
    default: return "unknown status";
  }
}

int f12int_create(f12int_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream) {
  if (!out) return F12INT_EINVAL;
  *out = nullptr;
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return F12INT_EINVAL;
  CK(cudaSetDevice(device));
  f12int_ctx *ctx = new (std::nothrow) f12int_ctx();
  if (!ctx) return F12INT_ENOMEM;
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  ctx->stream = (cudaStream_t)cuda_stream;
  int rc = upload_constants();
  if (rc == F12INT_OK) rc = dalloc(ctx, &ctx->d_status, sizeof(unsigned int));
  if (rc == F12INT_OK && cudaMemset(ctx->d_status, 0, sizeof(unsigned int)) != cudaSuccess) rc = F12INT_ECUDA;
  if (rc != F12INT_OK) {
    f12int_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return F12INT_OK;
}

static void engine_shutdown(f12int_ctx *ctx);
static bool engine_idle(f12int_ctx *ctx);
static void engine_factor_changed(f12int_ctx *ctx);

int f12int_destroy(f12int_ctx *ctx) {
  if (!ctx) return F12INT_EINVAL;
  cudaSetDevice(ctx->device);
  engine_shutdown(ctx);
  cudaDeviceSynchronize();
  for (auto &b : ctx->bases) {
    cudaFree(b.d_shell_l);
    cudaFree(b.d_centers);
    cudaFree(b.d_pair_start);
    cudaFree(b.d_pp_p);
    cudaFree(b.d_pp_P);
    cudaFree(b.d_pp_ab);
    cudaFree(b.d_epool);
    cudaFree(b.d_pp_eoff);
    for (int c = 0; c < 7; ++c) cudaFree(b.d_qprim[c]);
  }
  cudaFree(ctx->d_fam);
  cudaFree(ctx->d_coef);
  cudaFree(ctx->d_grp);
  cudaFree(ctx->d_jtab);
  cudaFree(ctx->d_kgrow);
  cudaFree(ctx->d_pqoff);
  cudaFree(ctx->d_keys);
  cudaFree(ctx->d_order);
  cudaFree(ctx->d_hist);
  cudaFree(ctx->d_part);
  cudaFree(ctx->d_qperm);
  cudaFree(ctx->d_operm);
  cudaFree(ctx->d_tasks);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_fma);
  for (auto &e : ctx->ev_pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  delete ctx;
  return F12INT_OK;
}

int64_t f12int_launch_count(const f12int_ctx *ctx) { return ctx ? ctx->launches : -1; }

int f12int_set_timing(f12int_ctx *ctx, int on) {
  if (!ctx) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  if (on && !ctx->d_fma) {
    int rc = dalloc(ctx, &ctx->d_fma, 2 * sizeof(unsigned long long));
    if (rc != F12INT_OK) return rc;
    CK(cudaMemset(ctx->d_fma, 0, 2 * sizeof(unsigned long long)));
  }
  ctx->timing = on != 0;
  return F12INT_OK;
}

int f12int_kernel_stats(f12int_ctx *ctx, int reset, double *stats) {
  if (!ctx || !stats) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  collect_events(ctx);
  unsigned long long cnt[2] = {0, 0};
  if (ctx->d_fma) CK(cudaMemcpy(cnt, ctx->d_fma, sizeof(cnt), cudaMemcpyDeviceToHost));
  stats[0] = ctx->aux_ms;
  stats[1] = (double)ctx->aux_launches;
  stats[2] = ctx->contract_ms;
  stats[3] = (double)ctx->contract_launches;
  stats[4] = 2.0 * (double)cnt[0];
  stats[5] = (double)cnt[1];
  if (reset) {
    ctx->aux_ms = ctx->contract_ms = 0.0;
    ctx->aux_launches = ctx->contract_launches = 0;
    if (ctx->d_fma) CK(cudaMemset(ctx->d_fma, 0, sizeof(cnt)));
  }
  return F12INT_OK;
}

int f12int_host_stats(f12int_ctx *ctx, int reset, double *stats) {
  if (!ctx || !stats) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  stats[0] = ctx->plan_ms;
  stats[1] = (double)ctx->plan_calls;
  if (reset) {
    ctx->plan_ms = 0.0;
    ctx->plan_calls = 0;
  }
  return F12INT_OK;
}

int f12int_set_series_cap(f12int_ctx *ctx, int kmax) {
  if (!ctx || kmax < 0) return F12INT_EINVAL;
  if (!engine_idle(ctx)) return F12INT_EINVAL;   // submitted requests use the current tables
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->series_cap = kmax == 0 ? KMAX : std::min(kmax, KMAX);
  ctx->tables.kcap = ctx->series_cap;
  engine_factor_changed(ctx);
  return F12INT_OK;
}

int f12int_device_status(f12int_ctx *ctx) {
  if (!ctx) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  unsigned int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned int), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return h ? F12INT_EDEVICE : F12INT_OK;
}

}  // extern "C"

// x^{2l+2} (D_r^l k)(x) of a kernel from its families.
static double kernel_radial_value(const f12::TermList &kt, int l, double x) {
  std::vector<f12::Family> fl = f12::families(kt);
  double s = 0.0;
  for (const f12::Family &fam0 : fl) {
    f12::Family cur = fam0;
    for (int k = 0; k < l; ++k) cur = f12::radial_derivative(cur);
    // x^{2l+2} * sum_j P_j x^{a0 - 2l + j} e^{b x - g x^2}, with a0 the original lowest power
    double poly = 0.0;
    for (size_t j = cur.poly.size(); j-- > 0;) poly = poly * x + cur.poly[j];
    s += poly * std::pow(x, fam0.a0 + 2.0) * std::exp(fam0.b * x - fam0.g * x * x);
  }
  return s;
}

extern "C" {

int f12int_kernel_radial(int cls, const f12int_factor *f, const f12int_factor *fprime, int l, double x,
                         double *value) {
  if (!f || !value || cls < 1 || cls > 6 || l < 0 || l > LAUX || !(x > 0.0)) return F12INT_EINVAL;
  const f12int_factor &fp = fprime ? *fprime : *f;
  int rc = check_factor(*f);
  if (rc == F12INT_OK) rc = check_factor(fp);
  if (rc != F12INT_OK) return rc;
  f12::Factor F1{f->c0, f->rho, f->B, f->mu, f->n}, F2{fp.c0, fp.rho, fp.B, fp.mu, fp.n};
  *value = kernel_radial_value(f12::kernel_terms(cls, F1, F2), l, x);
  return F12INT_OK;
}

}  // extern "C"

static int factor_class_flags(const f12::TermList &T1, const f12::TermList &T2, int *flags) {
  f12::TermList kt[NCLASS];
  for (int cls = 1; cls <= 6; ++cls)
    if (cls != 5) kt[cls] = f12::kernel_terms(cls, T1, T2);
  ClassTables ct;
  if (!build_class_tables(kt, ct)) return F12INT_EDOMAIN;
  flags[0] = 0;
  for (int c = 1; c <= 6; ++c) flags[c] = ct.supported[c] ? (ct.quad[c] ? 3 : 1) : 0;
  return F12INT_OK;
}

extern "C" {

int f12int_factor_classes(const f12int_factor *f, const f12int_factor *fprime, int *flags) {
  if (!f || !flags) return F12INT_EINVAL;
  const f12int_factor &fp = fprime ? *fprime : *f;
  int rc = check_factor(*f);
  if (rc == F12INT_OK) rc = check_factor(fp);
  if (rc != F12INT_OK) return rc;
  f12::Factor F1{f->c0, f->rho, f->B, f->mu, f->n}, F2{fp.c0, fp.rho, fp.B, fp.mu, fp.n};
  return factor_class_flags(f12::factor_terms(F1), f12::factor_terms(F2), flags);
}

int f12int_factor_classes_terms(const f12int_term *f, int nf, const f12int_term *fprime, int nfp, int *flags) {
  if (!flags) return F12INT_EINVAL;
  f12::TermList T1, T2;
  int rc = check_terms(f, nf, T1);
  if (rc == F12INT_OK) rc = fprime ? check_terms(fprime, nfp, T2) : (T2 = T1, F12INT_OK);
  if (rc != F12INT_OK) return rc;
  return factor_class_flags(T1, T2, flags);
}

int f12int_kernel_radial_terms(int cls, const f12int_term *f, int nf, const f12int_term *fprime, int nfp, int l,
                               double x, double *value) {
  if (!value || cls < 1 || cls > 6 || l < 0 || l > LAUX || !(x > 0.0)) return F12INT_EINVAL;
  f12::TermList T1, T2;
  int rc = check_terms(f, nf, T1);
  if (rc == F12INT_OK) rc = fprime ? check_terms(fprime, nfp, T2) : (T2 = T1, F12INT_OK);
  if (rc != F12INT_OK) return rc;
  *value = kernel_radial_value(f12::kernel_terms(cls, T1, T2), l, x);
  return F12INT_OK;
}

}  // extern "C"

// Screening estimate of a quartet: bound(ab) bound(cd) Gamma.  The diagonal
// blocks behind bound() sample the kernel at short range only; the F12
// kernels with B > 0 grow with r (Eq. rs12), so a quartet whose charge
// distributions lie R apart is larger by about the kernel's size there
// relative to short range.  With G(x) = max(1, max_{1 <= s <= x} |k(s)| /
// max_{1/2 <= s <= 3/2} |k(s)|) (G = 1 for 1/r), the overlap of the two
// distributions, exp(-xi w^2) at distance R + w, weighs the growth:
//   Gamma = max over w = 0, 0.5, .., 3 (in units of 1/sqrt(xi)) of
//           G(R + w) exp(-xi w^2),
// with R and xi = pq/(p+q) from each pair's most diffuse primitive pair.
// I5 (whose kinetic transform raises a quartet by about the bra exponents
// over the I3 diagonal it borrows) and I6 (whose f_r f'_r diagonal can cancel
// at short range) carry a further factor 8; on the 12-atom s/p/d sample the
// largest ratio of a quartet to its unscaled estimate was 55 (I5) and 49 (I6).
constexpr double kScreenSafety[7] = {1.0, 1.0, 1.0, 1.0, 1.0, 8.0, 8.0};
static std::vector<double> growth_table(const f12::TermList &t) {
  auto kval = [&](double x) {
    double v = 0.0;
    for (const f12::Term &u : t) v += u.c * std::pow(x, u.a) * std::exp(u.b * x - u.g * x * x);
    return std::fabs(v);
  };
  double kref = 0.0;
  for (double x = 0.5; x <= 1.5 + 1e-12; x += 0.01) kref = std::max(kref, kval(x));
  const int n = (int)(kGrowMax / kGrowStep) + 1;
  std::vector<double> g((size_t)n, 1.0);
  double run = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = i * kGrowStep;
    if (x >= 1.0) run = std::max(run, kval(x));
    g[i] = kref > 0.0 ? std::max(1.0, run / kref) : 1.0;
  }
  return g;
}

static double screen_estimate(const f12int_ctx *ctx, const f12int_ctx::BasisData &B, int cls, int a, int b, int c,
                              int d) {
  const std::vector<double> &pb = B.pair_bound[cls == 5 ? 3 : cls];
  const int ns = B.nshell;
  const size_t ab = (size_t)a * ns + b, cd = (size_t)c * ns + d;
  const double q = pb[ab] * pb[cd];
  const std::vector<double> &g = ctx->kgrow[cls];
  if (q == 0.0 || g.empty()) return q * kScreenSafety[cls];
  double r2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double dx = B.pair_cen[3 * ab + k] - B.pair_cen[3 * cd + k];
    r2 += dx * dx;
  }
  const double p = B.pair_pmin[ab], qq = B.pair_pmin[cd];
  const double xi = p * qq / (p + qq), R = std::sqrt(r2), w1 = 1.0 / std::sqrt(xi);
  double gam = 1.0;
  for (int k = 0; k <= 6; ++k) {
    const double w = 0.5 * k * w1;
    const size_t i = std::min(g.size() - 1, (size_t)((R + w) / kGrowStep) + 1);
    gam = std::max(gam, g[i] * std::exp(-xi * w * w));
  }
  return q * gam * kScreenSafety[cls];
}

// The part of f12int_set_factor(_terms) after validation: kernels, families,
// upload, and the bounds and schedules that depend on the factor.
static int set_factor_lists(f12int_ctx *ctx, const f12::TermList &T1, const f12::TermList &T2) {
  if (!engine_idle(ctx)) return F12INT_EINVAL;   // submitted requests still use the current factor
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  int rc = F12INT_OK;
  f12::TermList kt[NCLASS];
  for (int cls = 1; cls <= 6; ++cls)
    if (cls != 5) kt[cls] = f12::kernel_terms(cls, T1, T2);
  ClassTables ct;
  if (!build_class_tables(kt, ct)) return F12INT_EDOMAIN;
  const std::vector<FamDev> &fams = ct.fams;
  const std::vector<double> &coef = ct.coef;
  Tables T{};
  for (int c = 0; c < NCLASS; ++c) {
    T.nfam[c] = ct.nfam[c];
    T.fam0[c] = ct.fam0[c];
  }
  // upload
  dfree(ctx, ctx->d_fam, ctx->fam_bytes);
  dfree(ctx, ctx->d_coef, ctx->coef_bytes);
  dfree(ctx, ctx->d_grp, ctx->grp_bytes);
  dfree(ctx, ctx->d_jtab, ctx->jtab_bytes);
  ctx->d_grp = nullptr;
  ctx->d_jtab = nullptr;
  ctx->fam_bytes = fams.size() * sizeof(FamDev);
  ctx->coef_bytes = coef.size() * sizeof(double);
  ctx->grp_bytes = ct.groups.size() * sizeof(GroupDev);
  ctx->jtab_bytes = ct.jtab.size() * sizeof(double);
  rc = dalloc(ctx, &ctx->d_fam, ctx->fam_bytes);
  if (rc == F12INT_OK) rc = dalloc(ctx, &ctx->d_coef, ctx->coef_bytes);
  if (rc == F12INT_OK && ctx->grp_bytes) rc = dalloc(ctx, &ctx->d_grp, ctx->grp_bytes);
  if (rc == F12INT_OK && ctx->jtab_bytes) rc = dalloc(ctx, &ctx->d_jtab, ctx->jtab_bytes);
  if (rc != F12INT_OK) return rc;
  CK(cudaMemcpy(ctx->d_fam, fams.data(), ctx->fam_bytes, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_coef, coef.data(), ctx->coef_bytes, cudaMemcpyHostToDevice));
  if (ctx->grp_bytes)
    CK(cudaMemcpy(ctx->d_grp, ct.groups.data(), ctx->grp_bytes, cudaMemcpyHostToDevice));
  if (ctx->jtab_bytes)
    CK(cudaMemcpy(ctx->d_jtab, ct.jtab.data(), ctx->jtab_bytes, cudaMemcpyHostToDevice));
  T.fam = ctx->d_fam;
  T.coef = ctx->d_coef;
  T.grp = ctx->d_grp;
  T.jtab = ctx->d_jtab;
  T.kcap = ctx->series_cap;
  ctx->tables = T;
  for (int c = 1; c <= 6; ++c) {
    ctx->cls_ok[c] = ct.supported[c];
    ctx->cls_quad[c] = ct.quad[c];
  }
  for (auto &b : ctx->bases)   // the primitive bounds depend on the factor
    for (int c = 0; c < 7; ++c)
      if (b.d_qprim[c]) {
        cudaFree(b.d_qprim[c]);
        b.d_qprim[c] = nullptr;
      }
  for (auto &b : ctx->bases)   // and so do the shell-pair bounds
    for (int c = 0; c < 7; ++c) b.pair_bound[c].clear();
  for (int c = 1; c <= 6; ++c) ctx->kgrow[c] = growth_table(kt[c == 5 ? 3 : c]);
  {
    dfree(ctx, ctx->d_kgrow, ctx->kgrow_bytes);
    ctx->d_kgrow = nullptr;
    ctx->kgrow_n = (int)ctx->kgrow[1].size();
    std::vector<double> all((size_t)7 * ctx->kgrow_n, 1.0);
    for (int c = 1; c <= 6; ++c) {
      ctx->grows[c] = false;
      for (int i = 0; i < ctx->kgrow_n; ++i) {
        all[(size_t)c * ctx->kgrow_n + i] = ctx->kgrow[c][i];
        ctx->grows[c] = ctx->grows[c] || ctx->kgrow[c][i] > 1.0;
      }
    }
    ctx->kgrow_bytes = sizeof(double) * all.size();
    rc = dalloc(ctx, &ctx->d_kgrow, ctx->kgrow_bytes);
    if (rc != F12INT_OK) return rc;
    CK(cudaMemcpy(ctx->d_kgrow, all.data(), ctx->kgrow_bytes, cudaMemcpyHostToDevice));
  }
  engine_factor_changed(ctx);
  ctx->factor_ready = true;
  return F12INT_OK;
}

extern "C" {

int f12int_set_factor(f12int_ctx *ctx, const f12int_factor *f, const f12int_factor *fprime) {
  if (!ctx || !f) return F12INT_EINVAL;
  const f12int_factor &fp = fprime ? *fprime : *f;
  int rc = check_factor(*f);
  if (rc == F12INT_OK) rc = check_factor(fp);
  if (rc != F12INT_OK) return rc;
  f12::Factor F1{f->c0, f->rho, f->B, f->mu, f->n}, F2{fp.c0, fp.rho, fp.B, fp.mu, fp.n};
  return set_factor_lists(ctx, f12::factor_terms(F1), f12::factor_terms(F2));
}

int f12int_set_factor_terms(f12int_ctx *ctx, const f12int_term *f, int nf, const f12int_term *fprime, int nfp) {
  if (!ctx) return F12INT_EINVAL;
  f12::TermList T1, T2;
  int rc = check_terms(f, nf, T1);
  if (rc == F12INT_OK) rc = fprime ? check_terms(fprime, nfp, T2) : (T2 = T1, F12INT_OK);
  if (rc != F12INT_OK) return rc;
  return set_factor_lists(ctx, T1, T2);
}

int f12int_set_basis(f12int_ctx *ctx, int nshell, const double *centers, const int *l, const int *nprim,
                     const double *exps, const double *coefs, int *basis_id) {
  if (!ctx || nshell <= 0 || !centers || !l || !nprim || !exps || !coefs || !basis_id) return F12INT_EINVAL;
  int nptot = 0;
  for (int i = 0; i < nshell; ++i) {
    if (l[i] < 0 || l[i] > LSH || nprim[i] < 1) return F12INT_EINVAL;
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(centers[3 * i + k])) return F12INT_EINVAL;
    nptot += nprim[i];
  }
  for (int i = 0; i < nptot; ++i)
    if (!(exps[i] > 0.0) || !std::isfinite(exps[i]) || !std::isfinite(coefs[i])) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  f12int_ctx::BasisData B;
  B.nshell = nshell;
  B.l.assign(l, l + nshell);
  B.nprim.assign(nprim, nprim + nshell);
  B.centers.assign(centers, centers + 3 * nshell);
  B.exps.assign(exps, exps + nptot);
  B.coefs.assign(coefs, coefs + nptot);
  std::vector<int> poff(nshell);
  for (int i = 0, o = 0; i < nshell; ++i) {
    poff[i] = o;
    o += nprim[i];
  }
  // primitive pairs of every ordered shell pair (i, j), i outer
  std::vector<int> sa, sb, pa, pb;
  std::vector<int64_t> eoff;
  B.pair_start.assign((size_t)nshell * nshell + 1, 0);
  int64_t epos = 0;
  for (int i = 0; i < nshell; ++i)
    for (int j = 0; j < nshell; ++j) {
      B.pair_start[(size_t)i * nshell + j] = (int)sa.size();
      int n1 = (l[i] + 1) * (l[j] + 1) * (l[i] + l[j] + 1);
      for (int x = 0; x < nprim[i]; ++x)
        for (int y = 0; y < nprim[j]; ++y) {
          sa.push_back(i);
          sb.push_back(j);
          pa.push_back(poff[i] + x);
          pb.push_back(poff[j] + y);
          eoff.push_back(epos);
          epos += 6 * n1;
        }
    }
  B.pair_start[(size_t)nshell * nshell] = (int)sa.size();
  const int npp = (int)sa.size();
  // most diffuse primitive pair of every shell pair (screening geometry)
  B.pair_cen.assign((size_t)nshell * nshell * 3, 0.0);
  B.pair_pmin.assign((size_t)nshell * nshell, 0.0);
  for (int i = 0; i < nshell; ++i)
    for (int j = 0; j < nshell; ++j) {
      double ea = exps[poff[i]], eb = exps[poff[j]];
      for (int x = 1; x < nprim[i]; ++x) ea = std::min(ea, exps[poff[i] + x]);
      for (int y = 1; y < nprim[j]; ++y) eb = std::min(eb, exps[poff[j] + y]);
      const size_t k = (size_t)i * nshell + j;
      B.pair_pmin[k] = ea + eb;
      for (int d = 0; d < 3; ++d)
        B.pair_cen[3 * k + d] = (ea * centers[3 * i + d] + eb * centers[3 * j + d]) / (ea + eb);
    }
  // device buffers
  int *d_sa = nullptr, *d_sb = nullptr, *d_pa = nullptr, *d_pb = nullptr;
  double *d_exps = nullptr, *d_coefs = nullptr;
  int rc = F12INT_OK;
  size_t bytes = 0;
  auto A = [&](auto **p, size_t n) {
    if (rc != F12INT_OK) return;
    rc = dalloc(ctx, p, n);
    bytes += n;
  };
  A(&B.d_shell_l, sizeof(int) * nshell);
  A(&B.d_centers, sizeof(double) * 3 * nshell);
  A(&B.d_pair_start, sizeof(int) * B.pair_start.size());
  A(&B.d_pp_p, sizeof(double) * npp);
  A(&B.d_pp_P, sizeof(double) * 6 * npp);
  A(&B.d_pp_ab, sizeof(double) * 2 * npp);
  A(&B.d_pp_eoff, sizeof(int64_t) * npp);
  A(&B.d_epool, sizeof(double) * std::max<int64_t>(epos, 1));
  B.bytes = bytes;
  size_t tmpb = 0;
  auto At = [&](auto **p, size_t n) {
    if (rc != F12INT_OK) return;
    rc = dalloc(ctx, p, n);
    tmpb += n;
  };
  At(&d_sa, sizeof(int) * npp);
  At(&d_sb, sizeof(int) * npp);
  At(&d_pa, sizeof(int) * npp);
  At(&d_pb, sizeof(int) * npp);
  At(&d_exps, sizeof(double) * nptot);
  At(&d_coefs, sizeof(double) * nptot);
  if (rc == F12INT_OK) {
    cudaStream_t st = ctx->stream;
    cudaMemcpyAsync(B.d_shell_l, l, sizeof(int) * nshell, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B.d_centers, centers, sizeof(double) * 3 * nshell, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B.d_pair_start, B.pair_start.data(), sizeof(int) * B.pair_start.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(B.d_pp_eoff, eoff.data(), sizeof(int64_t) * npp, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_sa, sa.data(), sizeof(int) * npp, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_sb, sb.data(), sizeof(int) * npp, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_pa, pa.data(), sizeof(int) * npp, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_pb, pb.data(), sizeof(int) * npp, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_exps, exps, sizeof(double) * nptot, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_coefs, coefs, sizeof(double) * nptot, cudaMemcpyHostToDevice, st);
    int nb = (npp + 127) / 128;
    k_build_pairs<<<nb, 128, 0, st>>>(npp, d_sa, d_sb, d_pa, d_pb, B.d_centers, B.d_shell_l, d_exps, d_coefs,
                                      B.d_pp_p, B.d_pp_P, B.d_pp_ab, B.d_pp_eoff, B.d_epool);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  dfree(ctx, d_sa, sizeof(int) * npp);
  dfree(ctx, d_sb, sizeof(int) * npp);
  dfree(ctx, d_pa, sizeof(int) * npp);
  dfree(ctx, d_pb, sizeof(int) * npp);
  dfree(ctx, d_exps, sizeof(double) * nptot);
  dfree(ctx, d_coefs, sizeof(double) * nptot);
  if (rc != F12INT_OK) {
    cudaFree(B.d_shell_l);
    cudaFree(B.d_centers);
    cudaFree(B.d_pair_start);
    cudaFree(B.d_pp_p);
    cudaFree(B.d_pp_P);
    cudaFree(B.d_pp_ab);
    cudaFree(B.d_pp_eoff);
    cudaFree(B.d_epool);
    ctx->used -= std::min(ctx->used, B.bytes);
    return rc;
  }
  ctx->bases.push_back(std::move(B));
  *basis_id = (int)ctx->bases.size() - 1;
  return F12INT_OK;
}

static int ensure_buf(f12int_ctx *ctx, void **p, size_t *cap, size_t bytes) {
  if (*cap >= bytes) return F12INT_OK;
  if (*p) {
    cudaFree(*p);
    ctx->used -= std::min(ctx->used, *cap);
    *p = nullptr;
    *cap = 0;
  }
  size_t want = std::max(bytes, (size_t)1 << 16);
  int rc = dalloc(ctx, (char **)p, want);
  if (rc == F12INT_OK) *cap = want;
  return rc;
}

// shared memory of a contraction block with nw warps and nsplit ket ranges
// (esz: bytes per element, 8 for FP64, 4 for the FP32 path)
static size_t contract_smem(int la, int lb, int lc, int ld, int cls, int nw, int nsplit, size_t esz = 8) {
  int ext = cls == 5 ? 2 : 0;
  int L = la + lb + lc + ld + ext;
  int nhL = nh_count(L), nhB = nh_count(la + lb + ext);
  int ncd = ncart(lc) * ncart(ld), nab = ncart(la) * ncart(lb);
  int jc = (ncd + nsplit - 1) / nsplit;
  size_t e3ab = (size_t)ne3_count(la, lb) * (cls == 5 ? 4 : 1);
  const int ne3cd = ne3_chunk_max(lc, ld, jc), ne3ab = ne3_count(la, lb);
  return esz * ((size_t)nw * contract_warp_doubles(nhL, nhB, jc, ne3cd, L) + (size_t)nab * jc + e3ab) +
         sizeof(int) * ((size_t)ne3cd + ne3ab);
}

struct ContractPlan {
  int nw, nsplit;
  size_t smem;
};

// Algorithmic FP64 flops per primitive quartet of a task that owns jc ket
// components: Hermite recursion (repeated by every task of a quartet), ket
// and bra steps (x4 for I5).
static double task_flops(int la, int lb, int lc, int ld, int cls, int jc) {
  const int ext = cls == 5 ? 2 : 0;
  const int L = la + lb + lc + ld + ext;
  const double r = 2.0 * (L + 1) * (L + 2) * (L + 3) * (L + 4) / 24.0;
  const double ket = 2.0 * nh_count(la + lb + ext) * nh_count(lc + ld) * jc;
  const double bra = 2.0 * ncart(la) * ncart(lb) * nh_count(la + lb) * jc * (cls == 5 ? 4 : 1);
  return r + ket + bra;
}

// Work one contraction block should carry at most: a quartet with more is
// split into more ket ranges than its shared memory needs, so that its
// primitive quartets do not keep one SM busy while the others idle.
constexpr double kTaskFlops = 5e7;

static bool valid_split(int ncd, int ns) {
  const int jc = (ncd + ns - 1) / ns;
  return (ncd + jc - 1) / jc == ns;   // no empty ranges
}

static int work_split(int la, int lb, int lc, int ld, int cls, int64_t nprimq, int ns_min,
                      double target = kTaskFlops) {
  const int ncd = ncart(lc) * ncart(ld);
  for (int ns = ns_min; ns <= ncd; ++ns) {
    if (!valid_split(ncd, ns)) continue;
    if ((double)nprimq * task_flops(la, lb, lc, ld, cls, (ncd + ns - 1) / ns) <= target) return ns;
  }
  return ncd;
}

// Warps and ket ranges per contraction block for a quartet of nprimq
// primitive quartets: 4 warps, else 2, on the whole ket; where neither fits
// in 200 KB of shared memory, the fewest ket ranges that fit with 4 warps,
// else 2, else 1; then more ranges while a block would exceed kTaskFlops.
// smem = 0 when nothing fits.
static ContractPlan contract_plan(int la, int lb, int lc, int ld, int cls, int64_t nprimq, size_t esz = 8) {
  const size_t cap = 200 * 1024;
  const int ncd = ncart(lc) * ncart(ld);
  int nw = 0, ns = 1;
  for (int w = BLOCK_CONTRACT / 32; w > 1 && !nw; w /= 2)
    if (contract_smem(la, lb, lc, ld, cls, w, 1, esz) <= cap) nw = w;
  for (int w = BLOCK_CONTRACT / 32; w >= 1 && !nw; w /= 2)
    for (int k = 2; k <= ncd && !nw; ++k)
      if (valid_split(ncd, k) && contract_smem(la, lb, lc, ld, cls, w, k, esz) <= cap) {
        nw = w;
        ns = k;
      }
  if (!nw) return ContractPlan{1, 1, 0};
  ns = work_split(la, lb, lc, ld, cls, nprimq, ns);
  return ContractPlan{nw, ns, contract_smem(la, lb, lc, ld, cls, nw, ns, esz)};
}

static std::pair<cudaEvent_t, cudaEvent_t> take_events(f12int_ctx *ctx) {
  if (!ctx->ev_pool.empty()) {
    auto e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
  cudaEventCreate(&e.first);
  cudaEventCreate(&e.second);
  return e;
}

// After the stream has drained: add the timed launches to the totals.
static void collect_events(f12int_ctx *ctx) {
  for (auto &e : ctx->ev_aux) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) ctx->aux_ms += ms;
    ctx->ev_pool.push_back(e);
  }
  for (auto &e : ctx->ev_con) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) ctx->contract_ms += ms;
    ctx->ev_pool.push_back(e);
  }
  ctx->ev_aux.clear();
  ctx->ev_con.clear();
}

// items of the auxiliary stage per chunk (bounds the scratch memory)
static const int64_t kItemChunk = (int64_t)32 << 20;
static const int kNKeys = MAXFAM * (LAUX + 1) * NZBIN + 1;

// Queue the auxiliary stage (classify, scan, scatter, evaluate) and the
// contraction for quartets [qa, qb) of the device list.
static int launch_chunk(f12int_ctx *ctx, const f12int_ctx::BasisData &B, int cls, const int32_t *d_quartets,
                        const int64_t *d_pqoff, int64_t n, int64_t qa, int64_t qb, int64_t pqa, int64_t pqb,
                        size_t smem, double *out_dev, const int64_t *offsets_dev, cudaStream_t st,
                        bool prim_screen = true) {
  PairView PV = pair_view(ctx, B, cls, B.prim_screen && prim_screen);
  QuartetView QV{d_quartets, d_pqoff, n, nullptr, nullptr, nullptr, nullptr};
  const int kcls = cls == 5 ? 3 : cls;
  const int nf = ctx->tables.nfam[kcls];
  const int64_t nitems = (pqb - pqa) * nf;
  if (nitems > 0) {
    int rc = ensure_buf(ctx, (void **)&ctx->d_keys, &ctx->keys_cap, sizeof(int) * nitems);
    if (rc == F12INT_OK) rc = ensure_buf(ctx, (void **)&ctx->d_order, &ctx->order_cap, sizeof(unsigned) * nitems);
    if (rc == F12INT_OK) rc = ensure_buf(ctx, (void **)&ctx->d_part, &ctx->part_cap, sizeof(double) * nitems * kPartPitch);
    if (rc == F12INT_OK) rc = ensure_buf(ctx, (void **)&ctx->d_hist, &ctx->hist_cap, sizeof(unsigned) * kNKeys);
    if (rc != F12INT_OK) return rc;
    CK(cudaMemsetAsync(ctx->d_hist, 0, sizeof(unsigned) * kNKeys, st));
    const unsigned nb = (unsigned)((nitems + BLOCK_AUX - 1) / BLOCK_AUX);
    const unsigned nbq = (unsigned)((pqb - pqa + BLOCK_AUX - 1) / BLOCK_AUX);
    k_items_classify<false><<<nbq, BLOCK_AUX, 0, st>>>(ctx->tables, PV, QV, cls, pqa, nitems, ctx->d_keys,
                                                       ctx->d_hist);
    k_items_scan<<<1, 1024, 0, st>>>(ctx->d_hist, kNKeys);
    k_items_scatter<<<nb, BLOCK_AUX, 0, st>>>(QV, nf, pqa, ctx->d_keys, ctx->d_hist, nitems, ctx->d_order);
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (ctx->timing) {
      ev = take_events(ctx);
      cudaEventRecord(ev.first, st);
    }
    k_items_eval<false><<<nb, BLOCK_AUX, 0, st>>>(ctx->tables, PV, QV, cls, pqa, nitems, ctx->d_order, ctx->d_keys,
                                                  ctx->d_part, ctx->d_status, ctx->timing ? ctx->d_fma : nullptr);
    if (ctx->cls_quad[cls]) {
      k_items_eval<false, true><<<nb, BLOCK_AUX, 0, st>>>(ctx->tables, PV, QV, cls, pqa, nitems, ctx->d_order,
                                                          ctx->d_keys, ctx->d_part, ctx->d_status,
                                                          ctx->timing ? ctx->d_fma : nullptr);
      ctx->launches++;
    }
    if (ctx->timing) {
      cudaEventRecord(ev.second, st);
      ctx->ev_aux.push_back(ev);
      ctx->aux_launches++;
    }
    ctx->launches += 4;
    CK(cudaGetLastError());
  }
  // contraction: quartets are ordered by decreasing shared-memory need; one
  // launch per tier of warps and shared memory (powers of two), one block per
  // (quartet, ket range) task
  std::vector<CTask> tasks;
  for (int64_t i = qa; i < qb; ++i)
    for (int sp = 0; sp < ctx->h_split[i]; ++sp) tasks.push_back(CTask{(int32_t)i, (int16_t)sp, (int16_t)ctx->h_split[i]});
  {
    int rc = ensure_buf(ctx, (void **)&ctx->d_tasks, &ctx->tasks_cap, sizeof(CTask) * tasks.size());
    if (rc != F12INT_OK) return rc;
    CK(cudaMemcpyAsync(ctx->d_tasks, tasks.data(), sizeof(CTask) * tasks.size(), cudaMemcpyHostToDevice, st));
  }
  int64_t t0 = 0;
  // the thin quartets are a suffix of the working order
  int64_t qthin = qb;
  while (qthin > qa && ctx->h_thin[qthin - 1] >= 0) --qthin;
  for (int64_t ra = qa; ra < qthin;) {
    const int nw = ctx->h_nw[ra];
    const char f32 = ctx->h_fp32[ra];
    const size_t sm0 = ctx->h_smem[ra];
    int64_t rb = ra + 1, nt = ctx->h_split[ra];
    while (rb < qthin && ctx->h_nw[rb] == nw && ctx->h_fp32[rb] == f32 && 2 * ctx->h_smem[rb] > sm0)
      nt += ctx->h_split[rb++];
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (ctx->timing) {
      ev = take_events(ctx);
      cudaEventRecord(ev.first, st);
    }
    if (f32) {
      if (sm0 > 48 * 1024)
        CK(cudaFuncSetAttribute(k_contract<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0));
      k_contract<false, float><<<(unsigned)nt, 32 * nw, sm0, st>>>(
          PV, QV, cls, nf, pqa, ctx->d_tasks + t0, nt, nullptr, ctx->d_keys, ctx->d_part, out_dev, offsets_dev,
          ctx->d_status,
          ctx->timing ? ctx->d_fma + 1 : nullptr);
    } else {
      if (sm0 > 48 * 1024)
        CK(cudaFuncSetAttribute(k_contract<false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm0));
      k_contract<false, double><<<(unsigned)nt, 32 * nw, sm0, st>>>(
          PV, QV, cls, nf, pqa, ctx->d_tasks + t0, nt, nullptr, ctx->d_keys, ctx->d_part, out_dev, offsets_dev,
          ctx->d_status,
          ctx->timing ? ctx->d_fma + 1 : nullptr);
    }
    t0 += nt;
    if (ctx->timing) {
      cudaEventRecord(ev.second, st);
      ctx->ev_con.push_back(ev);
      ctx->contract_launches++;
    }
    ctx->launches++;
    CK(cudaGetLastError());
    ra = rb;
  }
  // thin quartets: one launch per (la, lb, lc, ld), one warp per quartet
  for (int64_t ra = qthin; ra < qb;) {
    const int key = ctx->h_thin[ra];
    int64_t rb = ra + 1;
    while (rb < qb && ctx->h_thin[rb] == key) ++rb;
    const int64_t nt = rb - ra;   // one task each
    const ThinKernel kern = thin_kernel(key, cls == 5);
    if (!kern) return F12INT_EINVAL;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (ctx->timing) {
      ev = take_events(ctx);
      cudaEventRecord(ev.first, st);
    }
    kern<<<(unsigned)((nt + kThinWarps - 1) / kThinWarps), 32 * kThinWarps, 0, st>>>(
        PV, QV, nf, pqa, ctx->d_tasks + t0, nt, nullptr, ctx->d_keys, ctx->d_part, out_dev, offsets_dev,
        ctx->timing ? ctx->d_fma + 1 : nullptr);
    t0 += nt;
    if (ctx->timing) {
      cudaEventRecord(ev.second, st);
      ctx->ev_con.push_back(ev);
      ctx->contract_launches++;
    }
    ctx->launches++;
    CK(cudaGetLastError());
    ra = rb;
  }
  return F12INT_OK;
}

// Primitive Schwarz factors Q_ab = sqrt(max |(ab|k|ab)|) of every primitive
// pair of the basis for class cls (the I3 kernel for I5), from the diagonal
// blocks of a basis in which every primitive is its own shell.
static int ensure_prim_bounds(f12int_ctx *ctx, int basis_id, int cls) {
  std::lock_guard<std::recursive_mutex> blk(ctx->bounds_mu);
  {
    f12int_ctx::BasisData &B = ctx->bases[basis_id];
    if (!B.prim_screen || B.d_qprim[cls]) return F12INT_OK;
  }
  const int dcls = cls == 5 ? 3 : cls;
  std::vector<double> cen, ex, co;
  std::vector<int> ll, np1;
  std::vector<int> poff;
  int nprim_tot = 0;
  {
    const f12int_ctx::BasisData &B = ctx->bases[basis_id];
    for (int s = 0; s < B.nshell; ++s) {
      poff.push_back(nprim_tot);
      for (int k = 0; k < B.nprim[s]; ++k) {
        cen.insert(cen.end(), {B.centers[3 * s], B.centers[3 * s + 1], B.centers[3 * s + 2]});
        ll.push_back(B.l[s]);
        np1.push_back(1);
        ex.push_back(B.exps[nprim_tot]);
        co.push_back(B.coefs[nprim_tot]);
        ++nprim_tot;
      }
    }
  }
  int pid = -1;
  int rc = f12int_set_basis(ctx, nprim_tot, cen.data(), ll.data(), np1.data(), ex.data(), co.data(), &pid);
  if (rc != F12INT_OK) return rc;
  ctx->bases[pid].prim_screen = false;
  std::vector<int32_t> hq;
  std::vector<int64_t> off;
  int64_t tot = 0;
  for (int a = 0; a < nprim_tot; ++a)
    for (int b = 0; b <= a; ++b) {
      hq.insert(hq.end(), {a, b, a, b});
      off.push_back(tot);
      int nab = ncart(ll[a]) * ncart(ll[b]);
      tot += (int64_t)nab * nab;
    }
  const int64_t nq = (int64_t)off.size();
  int32_t *dq = nullptr;
  int64_t *doff = nullptr;
  double *dout = nullptr;
  std::vector<double> hout((size_t)tot);
  rc = dalloc(ctx, &dq, sizeof(int32_t) * hq.size());
  if (rc == F12INT_OK) rc = dalloc(ctx, &doff, sizeof(int64_t) * nq);
  if (rc == F12INT_OK) rc = dalloc(ctx, &dout, sizeof(double) * tot);
  cudaStream_t st = ctx->stream;
  if (rc == F12INT_OK &&
      (cudaMemcpyAsync(dq, hq.data(), sizeof(int32_t) * hq.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
       cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * nq, cudaMemcpyHostToDevice, st) != cudaSuccess))
    rc = F12INT_ECUDA;
  if (rc == F12INT_OK) rc = f12int_compute_class(ctx, pid, dcls, dq, nq, dout, doff, st);
  if (rc == F12INT_OK &&
      (cudaMemcpyAsync(hout.data(), dout, sizeof(double) * tot, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = F12INT_ECUDA;
  dfree(ctx, dq, sizeof(int32_t) * hq.size());
  dfree(ctx, doff, sizeof(int64_t) * nq);
  dfree(ctx, dout, sizeof(double) * tot);
  // release the per-primitive basis (it is the last one)
  {
    f12int_ctx::BasisData &P = ctx->bases[pid];
    cudaFree(P.d_shell_l);
    cudaFree(P.d_centers);
    cudaFree(P.d_pair_start);
    cudaFree(P.d_pp_p);
    cudaFree(P.d_pp_P);
    cudaFree(P.d_pp_ab);
    cudaFree(P.d_pp_eoff);
    cudaFree(P.d_epool);
    ctx->used -= std::min(ctx->used, P.bytes);
    if (pid == (int)ctx->bases.size() - 1) ctx->bases.pop_back();
  }
  if (rc != F12INT_OK) return rc;
  std::vector<double> qps((size_t)nprim_tot * nprim_tot, 0.0);
  int64_t k = 0;
  for (int a = 0; a < nprim_tot; ++a)
    for (int b = 0; b <= a; ++b, ++k) {
      int nab = ncart(ll[a]) * ncart(ll[b]);
      double m = 0.0;
      for (int64_t i = 0; i < (int64_t)nab * nab; ++i) m = std::max(m, std::fabs(hout[off[k] + i]));
      qps[(size_t)a * nprim_tot + b] = qps[(size_t)b * nprim_tot + a] = std::sqrt(m);
    }
  f12int_ctx::BasisData &B = ctx->bases[basis_id];
  const int npp = B.pair_start.back();
  std::vector<double> qpp((size_t)npp);
  for (int a = 0; a < B.nshell; ++a)
    for (int b = 0; b < B.nshell; ++b) {
      int i = B.pair_start[(size_t)a * B.nshell + b];
      for (int x = 0; x < B.nprim[a]; ++x)
        for (int y = 0; y < B.nprim[b]; ++y, ++i) qpp[i] = qps[(size_t)(poff[a] + x) * nprim_tot + poff[b] + y];
    }
  double *d = nullptr;
  rc = dalloc(ctx, &d, sizeof(double) * npp);
  if (rc != F12INT_OK) return rc;
  if (cudaMemcpy(d, qpp.data(), sizeof(double) * npp, cudaMemcpyHostToDevice) != cudaSuccess) {
    dfree(ctx, d, sizeof(double) * npp);
    return F12INT_ECUDA;
  }
  B.d_qprim[cls] = d;
  return F12INT_OK;
}

static int compute_class_impl(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets_dev, int64_t n,
                              double *out_dev, const int64_t *offsets_dev, void *cuda_stream, double fp32_below,
                              bool prim_screen = true);
static int ensure_pair_bounds(f12int_ctx *ctx, int basis_id, int cls);

int f12int_compute_class(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets_dev, int64_t n,
                         double *out_dev, const int64_t *offsets_dev, void *cuda_stream) {
  return compute_class_impl(ctx, basis_id, cls, quartets_dev, n, out_dev, offsets_dev, cuda_stream, 0.0);
}

int f12int_compute_class_mixed(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets_dev, int64_t n,
                               double *out_dev, const int64_t *offsets_dev, double fp32_below, void *cuda_stream) {
  if (!(fp32_below >= 0.0)) return F12INT_EINVAL;
  return compute_class_impl(ctx, basis_id, cls, quartets_dev, n, out_dev, offsets_dev, cuda_stream, fp32_below);
}

}  // extern "C"

static int compute_class_impl(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets_dev, int64_t n,
                              double *out_dev, const int64_t *offsets_dev, void *cuda_stream, double fp32_below,
                              bool prim_screen) {
  if (!ctx) return F12INT_EINVAL;
  if (cls < 1 || cls > 6 || n < 0) return F12INT_EINVAL;
  if (basis_id < 0 || basis_id >= (int)ctx->bases.size()) return F12INT_ENOTREADY;
  if (!ctx->factor_ready) return F12INT_ENOTREADY;
  if (!ctx->cls_ok[cls]) return F12INT_EDOMAIN;
  if (n == 0) return F12INT_OK;
  if (!quartets_dev || !out_dev || !offsets_dev) return F12INT_EINVAL;
  {
    int rc0 = ensure_prim_bounds(ctx, basis_id, cls);
    if (rc0 == F12INT_OK && fp32_below > 0.0) rc0 = ensure_pair_bounds(ctx, basis_id, cls);
    if (rc0 != F12INT_OK) return rc0;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  const f12int_ctx::BasisData &B = ctx->bases[basis_id];
  cudaStream_t st = pick_stream(ctx, cuda_stream);
  NvtxRange call_range("f12int.compute_class");
  const auto t_plan0 = std::chrono::steady_clock::now();
  std::unique_ptr<NvtxRange> plan_range(new NvtxRange("f12int.plan"));
  // quartet metadata: order by (la, lb, lc, ld), primitive-quartet offsets
  std::vector<int32_t> hq0((size_t)4 * n);
  std::vector<int64_t> ho0((size_t)n);
  CK(cudaMemcpyAsync(hq0.data(), quartets_dev, sizeof(int32_t) * 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ho0.data(), offsets_dev, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int ns = B.nshell;
  std::vector<int> key0((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *s = &hq0[4 * i];
    for (int k = 0; k < 4; ++k)
      if (s[k] < 0 || s[k] >= ns) return F12INT_EINVAL;
    key0[i] = (B.l[s[0]] << 6) | (B.l[s[1]] << 4) | (B.l[s[2]] << 2) | B.l[s[3]];
  }
  // Every quartet with the same (primitive quartets, FP32 or not, class key)
  // has the same plan: the distinct ones ("plan groups") are planned once,
  // ordered -- FP64 first, decreasing shared-memory need (a tier launches
  // with the need of its first quartet, so no later one may need more),
  // decreasing work per task (the longest blocks start first), class key --
  // and the quartets are placed group by group in their list order (a
  // counting sort: linear in n).
  struct PlanGroup {
    ContractPlan pl;
    double work;
    int64_t key;
    int64_t count, first;
    bool thin;   // contracted by k_contract_thin
  };
  std::vector<PlanGroup> groups;
  std::vector<int32_t> gid((size_t)n);
  {
    // open-addressing map from the group key to its index
    std::vector<int64_t> slot_key(4096, -1);
    std::vector<int32_t> slot_val(4096, -1);
    size_t mask = slot_key.size() - 1;
    const std::vector<double> *pb = fp32_below > 0.0 ? &B.pair_bound[cls == 5 ? 3 : cls] : nullptr;
    for (int64_t i = 0; i < n; ++i) {
      const int k = key0[i];
      const int32_t *s = &hq0[4 * i];
      const int64_t np = (int64_t)B.nprim[s[0]] * B.nprim[s[1]] * B.nprim[s[2]] * B.nprim[s[3]];
      // mixed path: FP32 Hermite recursion and contraction below the bound
      const int f32 = (pb && screen_estimate(ctx, B, cls, s[0], s[1], s[2], s[3]) < fp32_below) ? 1 : 0;
      const int64_t gk = (np << 9) | (f32 << 8) | k;
      size_t h = (size_t)((uint64_t)gk * 0x9E3779B97F4A7C15ull >> 40) & mask;
      while (slot_key[h] != -1 && slot_key[h] != gk) h = (h + 1) & mask;
      if (slot_key[h] == -1) {
        if (groups.size() * 2 >= slot_key.size()) {   // grow and rehash
          std::vector<int64_t> nk(slot_key.size() * 2, -1);
          std::vector<int32_t> nv(slot_key.size() * 2, -1);
          const size_t nm = nk.size() - 1;
          for (size_t t = 0; t < slot_key.size(); ++t)
            if (slot_key[t] != -1) {
              size_t g = (size_t)((uint64_t)slot_key[t] * 0x9E3779B97F4A7C15ull >> 40) & nm;
              while (nk[g] != -1) g = (g + 1) & nm;
              nk[g] = slot_key[t];
              nv[g] = slot_val[t];
            }
          slot_key.swap(nk);
          slot_val.swap(nv);
          mask = nm;
          h = (size_t)((uint64_t)gk * 0x9E3779B97F4A7C15ull >> 40) & mask;
          while (slot_key[h] != -1 && slot_key[h] != gk) h = (h + 1) & mask;
        }
        const int la = (k >> 6) & 3, lb = (k >> 4) & 3, lc = (k >> 2) & 3, ld = k & 3;
        PlanGroup g{};
        g.pl = contract_plan(la, lb, lc, ld, cls, np, f32 ? 4 : 8);
        if (g.pl.smem == 0) return F12INT_EINVAL;
        g.thin = thin_quartet(k, cls);
        if (g.thin) g.pl = ContractPlan{1, 1, 0};   // one warp of the thin kernel, no shared memory
        const int ncd = ncart(lc) * ncart(ld);
        g.work = (double)np * task_flops(la, lb, lc, ld, cls, (ncd + g.pl.nsplit - 1) / g.pl.nsplit);
        g.key = gk;
        slot_key[h] = gk;
        slot_val[h] = (int32_t)groups.size();
        groups.push_back(g);
      }
      const int32_t g = slot_val[h];
      gid[i] = g;
      groups[g].count++;
    }
  }
  {
    std::vector<int32_t> order(groups.size());
    for (size_t g = 0; g < groups.size(); ++g) order[g] = (int32_t)g;
    std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
      const PlanGroup &A = groups[x], &Bg = groups[y];
      if (A.thin != Bg.thin) return Bg.thin;   // the thin quartets last, by class key
      if (A.thin) return (A.key & 0xFF) < (Bg.key & 0xFF) || ((A.key & 0xFF) == (Bg.key & 0xFF) && A.key < Bg.key);
      const int fa = (int)((A.key >> 8) & 1), fb = (int)((Bg.key >> 8) & 1);
      if (fa != fb) return fa < fb;
      if (A.pl.smem != Bg.pl.smem) return A.pl.smem > Bg.pl.smem;
      if (A.work != Bg.work) return A.work > Bg.work;
      return (A.key & 0xFF) < (Bg.key & 0xFF) || ((A.key & 0xFF) == (Bg.key & 0xFF) && A.key < Bg.key);
    });
    int64_t run = 0;
    for (int32_t g : order) {
      groups[g].first = run;
      run += groups[g].count;
    }
  }
  std::vector<int64_t> perm((size_t)n);
  for (int64_t i = 0; i < n; ++i) perm[groups[gid[i]].first++] = i;
  std::vector<int32_t> hq((size_t)4 * n);
  std::vector<int64_t> ho((size_t)n);
  ctx->h_nw.resize((size_t)n);
  ctx->h_split.resize((size_t)n);
  ctx->h_smem.resize((size_t)n);
  ctx->h_fp32.resize((size_t)n);
  ctx->h_thin.resize((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t j = perm[i];
    for (int k = 0; k < 4; ++k) hq[4 * i + k] = hq0[4 * j + k];
    ho[i] = ho0[j];
    const PlanGroup &g = groups[gid[j]];
    ctx->h_nw[i] = g.pl.nw;
    ctx->h_split[i] = g.pl.nsplit;
    ctx->h_smem[i] = g.pl.smem;
    ctx->h_fp32[i] = (char)(g.thin ? 0 : (g.key >> 8) & 1);   // the thin kernel is FP64
    ctx->h_thin[i] = g.thin ? (int16_t)(g.key & 0xFF) : (int16_t)-1;
  }
  std::vector<int64_t> pqoff((size_t)n + 1);
  int64_t npq = 0;
  size_t smem = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *s = &hq[4 * i];
    pqoff[i] = npq;
    npq += (int64_t)B.nprim[s[0]] * B.nprim[s[1]] * B.nprim[s[2]] * B.nprim[s[3]];
    smem = std::max(smem, ctx->h_smem[i]);
  }
  pqoff[n] = npq;
  if (smem > 227 * 1024) return F12INT_EINVAL;
  int rc = ensure_buf(ctx, (void **)&ctx->d_pqoff, &ctx->pqoff_cap, sizeof(int64_t) * ((size_t)n + 1));
  if (rc == F12INT_OK) rc = ensure_buf(ctx, (void **)&ctx->d_qperm, &ctx->qperm_cap, sizeof(int32_t) * 4 * n);
  if (rc == F12INT_OK) rc = ensure_buf(ctx, (void **)&ctx->d_operm, &ctx->operm_cap, sizeof(int64_t) * n);
  if (rc != F12INT_OK) return rc;
  CK(cudaMemcpyAsync(ctx->d_pqoff, pqoff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_qperm, hq.data(), sizeof(int32_t) * 4 * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_operm, ho.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  const int kcls = cls == 5 ? 3 : cls;
  const int64_t nf = ctx->tables.nfam[kcls];
  const int64_t pq_chunk = std::max<int64_t>(1, kItemChunk / std::max<int64_t>(nf, 1));
  plan_range.reset();
  ctx->plan_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_plan0).count();
  ctx->plan_calls++;
  for (int64_t qa = 0; qa < n;) {
    int64_t qb = qa + 1;
    while (qb < n && pqoff[qb + 1] - pqoff[qa] <= pq_chunk) ++qb;
    rc = launch_chunk(ctx, B, cls, ctx->d_qperm, ctx->d_pqoff, n, qa, qb, pqoff[qa], pqoff[qb], smem, out_dev,
                      ctx->d_operm, st, prim_screen);
    if (rc != F12INT_OK) return rc;
    qa = qb;
  }
  // keep the host buffer alive until the copy has been consumed
  CK(cudaStreamSynchronize(st));
  if (ctx->timing) collect_events(ctx);
  return F12INT_OK;
}

extern "C" {

int f12int_aux(f12int_ctx *ctx, int cls, int64_t npts, const double *xi_dev, const double *D_dev, int nmax,
               double *out_dev, void *cuda_stream) {
  if (!ctx || cls < 1 || cls > 6 || npts < 0 || nmax < 0 || nmax > LAUX) return F12INT_EINVAL;
  if (!ctx->factor_ready) return F12INT_ENOTREADY;
  if (!ctx->cls_ok[cls]) return F12INT_EDOMAIN;
  if (npts == 0) return F12INT_OK;
  if (!xi_dev || !D_dev || !out_dev) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = pick_stream(ctx, cuda_stream);
  int64_t nb = (npts + BLOCK_AUX - 1) / BLOCK_AUX;
  k_aux_points<<<(unsigned)nb, BLOCK_AUX, 0, st>>>(ctx->tables, cls, npts, xi_dev, D_dev, nmax, out_dev,
                                                   ctx->d_status);
  ctx->launches++;
  CK(cudaGetLastError());
  return F12INT_OK;
}

// Shell-pair bounds bound(ab) = sqrt(max |(ab|k|ab)|) over the diagonal block
// (the I3 kernel for I5), cached per basis and class.
static int ensure_pair_bounds(f12int_ctx *ctx, int basis_id, int cls) {
  const int dcls = cls == 5 ? 3 : cls;
  std::lock_guard<std::recursive_mutex> blk(ctx->bounds_mu);
  if (!ctx->bases[basis_id].pair_bound[dcls].empty()) return F12INT_OK;
  const f12int_ctx::BasisData &B = ctx->bases[basis_id];
  const int ns = B.nshell;
  // diagonal blocks (ab|ab) for a >= b
  std::vector<int32_t> hq;
  std::vector<int64_t> off;
  int64_t tot = 0;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b <= a; ++b) {
      hq.insert(hq.end(), {a, b, a, b});
      off.push_back(tot);
      int nab = ncart(B.l[a]) * ncart(B.l[b]);
      tot += (int64_t)nab * nab;
    }
  const int64_t nq = (int64_t)off.size();
  int32_t *dq = nullptr;
  int64_t *doff = nullptr;
  double *dout = nullptr;
  int rc = dalloc(ctx, &dq, sizeof(int32_t) * hq.size());
  if (rc == F12INT_OK) rc = dalloc(ctx, &doff, sizeof(int64_t) * nq);
  if (rc == F12INT_OK) rc = dalloc(ctx, &dout, sizeof(double) * tot);
  std::vector<double> hout((size_t)tot);
  if (rc == F12INT_OK) {
    cudaStream_t st = ctx->stream;
    if (cudaMemcpyAsync(dq, hq.data(), sizeof(int32_t) * hq.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * nq, cudaMemcpyHostToDevice, st) != cudaSuccess)
      rc = F12INT_ECUDA;
    // the diagonal blocks themselves can be far below the primitive screen
    // (a pair's bound multiplies a partner's that may be large), so they are
    // computed without it
    if (rc == F12INT_OK)
      rc = compute_class_impl(ctx, basis_id, dcls, dq, nq, dout, doff, st, 0.0, /*prim_screen=*/false);
    if (rc == F12INT_OK &&
        (cudaMemcpyAsync(hout.data(), dout, sizeof(double) * tot, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
      rc = F12INT_ECUDA;
  }
  dfree(ctx, dq, sizeof(int32_t) * hq.size());
  dfree(ctx, doff, sizeof(int64_t) * nq);
  dfree(ctx, dout, sizeof(double) * tot);
  if (rc != F12INT_OK) return rc;
  std::vector<double> bound((size_t)ns * ns, 0.0);
  int64_t k = 0;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b <= a; ++b, ++k) {
      int nab = ncart(B.l[a]) * ncart(B.l[b]);
      double m = 0.0;
      for (int64_t i = 0; i < (int64_t)nab * nab; ++i) m = std::max(m, std::fabs(hout[off[k] + i]));
      bound[(size_t)a * ns + b] = bound[(size_t)b * ns + a] = std::sqrt(m);
    }
  ctx->bases[basis_id].pair_bound[dcls] = std::move(bound);
  return F12INT_OK;
}

int f12int_pair_bounds(f12int_ctx *ctx, int basis_id, int cls, double *bounds_out) {
  if (!ctx || cls < 1 || cls > 6 || !bounds_out) return F12INT_EINVAL;
  if (basis_id < 0 || basis_id >= (int)ctx->bases.size() || !ctx->factor_ready) return F12INT_ENOTREADY;
  int rc = ensure_pair_bounds(ctx, basis_id, cls);
  if (rc != F12INT_OK) return rc;
  const std::vector<double> &b = ctx->bases[basis_id].pair_bound[cls == 5 ? 3 : cls];
  std::memcpy(bounds_out, b.data(), sizeof(double) * b.size());
  return F12INT_OK;
}

int f12int_quartet_estimates(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets, int64_t n,
                             double *est_out) {
  if (!ctx || cls < 1 || cls > 6 || n < 0 || (n > 0 && (!quartets || !est_out))) return F12INT_EINVAL;
  if (basis_id < 0 || basis_id >= (int)ctx->bases.size() || !ctx->factor_ready) return F12INT_ENOTREADY;
  int rc = ensure_pair_bounds(ctx, basis_id, cls);
  if (rc != F12INT_OK) return rc;
  const f12int_ctx::BasisData &B = ctx->bases[basis_id];
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *q = quartets + 4 * i;
    for (int k = 0; k < 4; ++k)
      if (q[k] < 0 || q[k] >= B.nshell) return F12INT_EINVAL;
    est_out[i] = screen_estimate(ctx, B, cls, q[0], q[1], q[2], q[3]);
  }
  return F12INT_OK;
}

int f12int_screen(f12int_ctx *ctx, int basis_id, int cls, double thresh, int32_t *quartets_out, int64_t cap,
                  int64_t *n_out) {
  if (!ctx || cls < 1 || cls > 6 || !n_out || cap < 0 || (cap > 0 && !quartets_out)) return F12INT_EINVAL;
  if (basis_id < 0 || basis_id >= (int)ctx->bases.size() || !ctx->factor_ready) return F12INT_ENOTREADY;
  if (!(thresh >= 0.0)) return F12INT_EINVAL;
  int rc = ensure_pair_bounds(ctx, basis_id, cls);
  if (rc != F12INT_OK) return rc;
  const f12int_ctx::BasisData &B = ctx->bases[basis_id];
  const int ns = B.nshell;
  const std::vector<double> &bound = B.pair_bound[cls == 5 ? 3 : cls];
  std::vector<std::pair<int, int>> pairs;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b <= a; ++b) pairs.emplace_back(a, b);
  int64_t cnt = 0;
  const std::vector<double> &g = ctx->kgrow[cls];
  const double gmax = g.empty() ? 1.0 : g.back();   // G is non-decreasing
  for (size_t i = 0; i < pairs.size(); ++i) {
    size_t jend = (cls == 5) ? pairs.size() : i + 1;
    double bi = bound[(size_t)pairs[i].first * ns + pairs[i].second];
    for (size_t j = 0; j < jend; ++j) {
      double bj = bound[(size_t)pairs[j].first * ns + pairs[j].second];
      const double q = bi * bj;
      if (q >= thresh ||
          (q * gmax * kScreenSafety[cls] >= thresh &&
           screen_estimate(ctx, B, cls, pairs[i].first, pairs[i].second, pairs[j].first, pairs[j].second) >=
               thresh)) {
        if (cnt < cap) {
          quartets_out[4 * cnt] = pairs[i].first;
          quartets_out[4 * cnt + 1] = pairs[i].second;
          quartets_out[4 * cnt + 2] = pairs[j].first;
          quartets_out[4 * cnt + 3] = pairs[j].second;
        }
        ++cnt;
      }
    }
  }
  *n_out = cnt;
  return F12INT_OK;
}

}  // extern "C"

// ===================================================== static-scratch variant ==
// Callers that must not allocate device memory while they run (for example a
// host application that reserves all device memory up front for its own
// pool, or a latency-sensitive service in which the device-wide
// synchronisation of a cudaMalloc would stall work on other streams) use
// f12int_compute_class_static.  It runs the same kernels as
// f12int_compute_class but takes every scratch buffer from the file-scope
// array below, which each GPU that loads the library holds until exit.

#define F12INT_STATIC_SCRATCH_BYTES ((size_t)64 << 20)

static __device__ __align__(256) unsigned char g_static_scratch[F12INT_STATIC_SCRATCH_BYTES];

namespace {

// Device address of g_static_scratch, resolved once per device.  In host code
// the array's name is only a stand-in; the address must come from
// cudaGetSymbolAddress with the device current.
std::mutex g_static_mu;
void *g_static_addr[64] = {nullptr};

int static_scratch_address(int device, unsigned char **out) {
  if (device < 0 || device >= 64) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return F12INT_ECUDA;
    g_static_addr[device] = p;
  }
  *out = (unsigned char *)g_static_addr[device];
  return F12INT_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int f12int_compute_class_static(f12int_ctx *ctx, int basis_id, int cls, const int32_t *quartets_dev,
                                           int64_t n, double *out_dev, const int64_t *offsets_dev,
                                           void *cuda_stream) {
  if (!ctx) return F12INT_EINVAL;
  if (cls < 1 || cls > 6 || n < 0) return F12INT_EINVAL;
  if (basis_id < 0 || basis_id >= (int)ctx->bases.size()) return F12INT_ENOTREADY;
  if (!ctx->factor_ready) return F12INT_ENOTREADY;
  if (!ctx->cls_ok[cls]) return F12INT_EDOMAIN;
  if (n == 0) return F12INT_OK;
  if (!quartets_dev || !out_dev || !offsets_dev) return F12INT_EINVAL;
  // a first bound on the list length, before anything is read back
  const size_t per_quartet = sizeof(int32_t) * 4 + sizeof(int64_t) * 2 + sizeof(CTask);
  if ((size_t)n > F12INT_STATIC_SCRATCH_BYTES / per_quartet) return F12INT_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  unsigned char *base = nullptr;
  int rc = static_scratch_address(ctx->device, &base);
  if (rc != F12INT_OK) return rc;
  const size_t item_bytes = sizeof(int) + sizeof(unsigned) + sizeof(double) * kPartPitch;

  const f12int_ctx::BasisData &B = ctx->bases[basis_id];
  cudaStream_t st = pick_stream(ctx, cuda_stream);
  std::vector<int32_t> hq0((size_t)4 * n);
  std::vector<int64_t> ho0((size_t)n);
  CK(cudaMemcpyAsync(hq0.data(), quartets_dev, sizeof(int32_t) * 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ho0.data(), offsets_dev, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int ns = B.nshell;
  std::vector<size_t> sm0((size_t)n);
  std::vector<int> nw0((size_t)n), sp0((size_t)n), key0((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t *s = &hq0[4 * i];
    for (int k = 0; k < 4; ++k)
      if (s[k] < 0 || s[k] >= ns) return F12INT_EINVAL;
    key0[i] = (B.l[s[0]] << 6) | (B.l[s[1]] << 4) | (B.l[s[2]] << 2) | B.l[s[3]];
    const ContractPlan pl = contract_plan(B.l[s[0]], B.l[s[1]], B.l[s[2]], B.l[s[3]], cls,
                                          (int64_t)B.nprim[s[0]] * B.nprim[s[1]] * B.nprim[s[2]] * B.nprim[s[3]]);
    if (pl.smem == 0 || pl.smem > 227 * 1024) return F12INT_EINVAL;
    nw0[i] = pl.nw;
    sp0[i] = pl.nsplit;
    sm0[i] = pl.smem;
    if (thin_quartet(key0[i], cls)) {   // k_contract_thin: sorted last (no shared memory), by key
      nw0[i] = 1;
      sp0[i] = 1;
      sm0[i] = 0;
    }
  }
  std::vector<int64_t> perm((size_t)n);
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int64_t x, int64_t y) {
    if (sm0[x] != sm0[y]) return sm0[x] > sm0[y];
    return key0[x] < key0[y];
  });
  std::vector<int32_t> hq((size_t)4 * n);
  std::vector<int64_t> ho((size_t)n), pqoff((size_t)n + 1);
  std::vector<int> hnw((size_t)n), hsp((size_t)n);
  std::vector<size_t> hsm((size_t)n);
  int64_t npq = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 4; ++k) hq[4 * i + k] = hq0[4 * perm[i] + k];
    ho[i] = ho0[perm[i]];
    hnw[i] = nw0[perm[i]];
    hsp[i] = sp0[perm[i]];
    hsm[i] = sm0[perm[i]];
    const int32_t *s = &hq[4 * i];
    pqoff[i] = npq;
    npq += (int64_t)B.nprim[s[0]] * B.nprim[s[1]] * B.nprim[s[2]] * B.nprim[s[3]];
  }
  pqoff[n] = npq;
  // contraction tasks (one per quartet and ket range), then the work items
  std::vector<CTask> tasks;
  for (int64_t i = 0; i < n; ++i)
    for (int sp = 0; sp < hsp[i]; ++sp) tasks.push_back(CTask{(int32_t)i, (int16_t)sp, (int16_t)hsp[i]});
  std::vector<int64_t> tfirst((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; ++i) tfirst[i + 1] = tfirst[i] + hsp[i];
  // layout of the array: quartets, offsets and primitive offsets in the
  // working order, the key histogram and the task list (all sized exactly
  // now), then the work items of one chunk.  Every size check happens here,
  // before anything is queued, so that an F12INT_EINVAL leaves the array and
  // the output untouched.
  int32_t *d_q = (int32_t *)base;
  int64_t *d_o = (int64_t *)(base + align256(sizeof(int32_t) * 4 * (size_t)n));
  int64_t *d_pq = (int64_t *)((unsigned char *)d_o + align256(sizeof(int64_t) * (size_t)n));
  unsigned *d_hist = (unsigned *)((unsigned char *)d_pq + align256(sizeof(int64_t) * ((size_t)n + 1)));
  CTask *d_tk = (CTask *)((unsigned char *)d_hist + align256(sizeof(unsigned) * kNKeys));
  unsigned char *items_base = (unsigned char *)d_tk + align256(sizeof(CTask) * tasks.size());
  const size_t used_fixed = (size_t)(items_base - base);
  if (used_fixed + 3 * 256 + item_bytes > F12INT_STATIC_SCRATCH_BYTES) return F12INT_EINVAL;
  const int64_t max_items = (int64_t)((F12INT_STATIC_SCRATCH_BYTES - used_fixed - 3 * 256) / item_bytes);
  const int kcls = cls == 5 ? 3 : cls;
  const int nf = ctx->tables.nfam[kcls];
  const int64_t pq_chunk = std::max<int64_t>(1, max_items / std::max(nf, 1));
  for (int64_t i = 0; i < n; ++i)
    if (pqoff[i + 1] - pqoff[i] > pq_chunk) return F12INT_EINVAL;   // one quartet larger than the scratch
  CK(cudaMemcpyAsync(d_tk, tasks.data(), sizeof(CTask) * tasks.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_q, hq.data(), sizeof(int32_t) * 4 * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_o, ho.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_pq, pqoff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));

  // the primitive screen of f12int_compute_class when its table for this
  // (basis, class) exists already (building it would allocate); without it
  // every primitive quartet is evaluated
  PairView PV = pair_view(ctx, B, cls, B.prim_screen);
  QuartetView QV{d_q, d_pq, n, nullptr, nullptr, nullptr, nullptr};
  int rc_launch = F12INT_OK;
  for (int64_t qa = 0; qa < n && rc_launch == F12INT_OK;) {
    int64_t qb = qa + 1;
    while (qb < n && pqoff[qb + 1] - pqoff[qa] <= pq_chunk) ++qb;
    const int64_t pqa = pqoff[qa], nitems = (pqoff[qb] - pqa) * nf;
    int *d_keys = (int *)items_base;
    unsigned *d_order = (unsigned *)(items_base + align256(sizeof(int) * (size_t)nitems));
    double *d_part = (double *)((unsigned char *)d_order + align256(sizeof(unsigned) * (size_t)nitems));
    if (nitems > 0) {
      // the histogram must start at zero on every call: the array keeps the
      // previous call's contents
      if (cudaMemsetAsync(d_hist, 0, sizeof(unsigned) * kNKeys, st) != cudaSuccess) {
        rc_launch = F12INT_ECUDA;
        break;
      }
      const unsigned nb = (unsigned)((nitems + BLOCK_AUX - 1) / BLOCK_AUX);
      const unsigned nbq = (unsigned)((pqoff[qb] - pqa + BLOCK_AUX - 1) / BLOCK_AUX);
      k_items_classify<false><<<nbq, BLOCK_AUX, 0, st>>>(ctx->tables, PV, QV, cls, pqa, nitems, d_keys, d_hist);
      k_items_scan<<<1, 1024, 0, st>>>(d_hist, kNKeys);
      k_items_scatter<<<nb, BLOCK_AUX, 0, st>>>(QV, nf, pqa, d_keys, d_hist, nitems, d_order);
      k_items_eval<false><<<nb, BLOCK_AUX, 0, st>>>(ctx->tables, PV, QV, cls, pqa, nitems, d_order, d_keys, d_part,
                                                    ctx->d_status, nullptr);
      ctx->launches += 4;
      if (ctx->cls_quad[cls]) {
        k_items_eval<false, true><<<nb, BLOCK_AUX, 0, st>>>(ctx->tables, PV, QV, cls, pqa, nitems, d_order, d_keys,
                                                            d_part, ctx->d_status, nullptr);
        ctx->launches++;
      }
      if (cudaGetLastError() != cudaSuccess) rc_launch = F12INT_ECUDA;
    }
    for (int64_t ra = qa; ra < qb && rc_launch == F12INT_OK;) {
      const int nwr = hnw[ra];
      const size_t smr = hsm[ra];
      int64_t rb = ra + 1;
      if (smr == 0) {   // thin quartets: one launch per class key
        const int key = (B.l[hq[4 * ra]] << 6) | (B.l[hq[4 * ra + 1]] << 4) | (B.l[hq[4 * ra + 2]] << 2) |
                        B.l[hq[4 * ra + 3]];
        auto key_of = [&](int64_t i) {
          return (B.l[hq[4 * i]] << 6) | (B.l[hq[4 * i + 1]] << 4) | (B.l[hq[4 * i + 2]] << 2) | B.l[hq[4 * i + 3]];
        };
        while (rb < qb && hsm[rb] == 0 && key_of(rb) == key) ++rb;
        const int64_t nt = tfirst[rb] - tfirst[ra];
        const ThinKernel kern = thin_kernel(key, cls == 5);
        if (!kern) {
          rc_launch = F12INT_EINVAL;
          break;
        }
        kern<<<(unsigned)((nt + kThinWarps - 1) / kThinWarps), 32 * kThinWarps, 0, st>>>(
            PV, QV, nf, pqa, d_tk + tfirst[ra], nt, nullptr, d_keys, d_part, out_dev, d_o, nullptr);
        ctx->launches++;
        if (cudaGetLastError() != cudaSuccess) rc_launch = F12INT_ECUDA;
        ra = rb;
        continue;
      }
      while (rb < qb && hnw[rb] == nwr && 2 * hsm[rb] > smr) ++rb;
      const int64_t nt = tfirst[rb] - tfirst[ra];
      if (smr > 48 * 1024 &&
          cudaFuncSetAttribute(k_contract<false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr) !=
              cudaSuccess) {
        rc_launch = F12INT_ECUDA;
        break;
      }
      k_contract<false, double><<<(unsigned)nt, 32 * nwr, smr, st>>>(PV, QV, cls, nf, pqa, d_tk + tfirst[ra], nt, nullptr,
                                                                     d_keys, d_part, out_dev, d_o, ctx->d_status, nullptr);
      ctx->launches++;
      if (cudaGetLastError() != cudaSuccess) rc_launch = F12INT_ECUDA;
      ra = rb;
    }
    qa = qb;
  }
  // the host vectors above stay alive until the queued copies are consumed,
  // and on an error nothing of this call is still running when it returns
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc_launch != F12INT_OK) return rc_launch;
  if (e != cudaSuccess) return cuda_fail(e);
  return F12INT_OK;
}

#include "engine.cuh"
