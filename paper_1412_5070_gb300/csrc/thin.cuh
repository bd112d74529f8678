// thin.cuh -- the thin contraction kernel template, instantiated by
// thin_inst.cu in seven parts (seven objects compiled in parallel with the
// rest of the library).
#pragma once

#include "kernel_common.cuh"

namespace f12k {

// ---------------------------------------------------- thin contraction --
// Quartets of low total order (L = la+lb+lc+ld <= 3, and for I5 L <= 2;
// FP64): one warp takes a whole shell quartet and each lane one primitive
// quartet at a time (the general kernel would keep most of its lanes idle on
// them: 31 of 32 on an (ss|ss) quartet).  A lane forms g_n, R_tuv and the E
// products in registers and accumulates every element of the block (Eq. ii,
// bra sign (-1)^{t+u+v}; for I5 Eq. I5byI3_ with the second coefficient -1,
// as the general kernel); the lanes' sums are then added by a fixed
// butterfly, so the result does not depend on scheduling.

__host__ __device__ constexpr int cart_i(int l, int k) {   // x exponent of component k of shell l
  int n = 0;
  for (int i = l; i >= 0; --i)
    for (int j = l - i; j >= 0; --j, ++n)
      if (n == k) return i;
  return 0;
}
__host__ __device__ constexpr int cart_j(int l, int k) {   // y exponent
  int n = 0;
  for (int i = l; i >= 0; --i)
    for (int j = l - i; j >= 0; --j, ++n)
      if (n == k) return j;
  return 0;
}

// One shell quartet q (index into the list) by the calling warp; its block
// goes to o.
template <int LA, int LB, int LC, int LD, bool I5>
__device__ __forceinline__ void thin_quartet_body(const PairView &PV, const QuartetView &QV, int nf, int64_t pq0,
                                                  int64_t q, const int *keys, const double *part, double *out_q,
                                                  unsigned long long *flops_total) {
  constexpr int EXT = I5 ? 2 : 0;
  constexpr int L = LA + LB + LC + LD + EXT;   // highest order of g_n and R
  constexpr int NA = (LA + 1) * (LA + 2) / 2, NB = (LB + 1) * (LB + 2) / 2;
  constexpr int NC = (LC + 1) * (LC + 2) / 2, ND = (LD + 1) * (LD + 2) / 2;
  constexpr int NE = NA * NB * NC * ND;
  constexpr int NTAB = LA + LB + 1, NTCD = LC + LD + 1;
  constexpr int N1AB = (LA + 1) * (LB + 1) * NTAB, N1CD = (LC + 1) * (LD + 1) * NTCD;
  constexpr int NH = (L + 1) * (L + 2) * (L + 3) / 6;
  const int lane = threadIdx.x & 31;
  const int32_t *s = QV.quartets + 4 * q;
  const int ns = PV.nshell;
  const int ab = s[0] * ns + s[1], cd = s[2] * ns + s[3];
  const int ab0 = PV.pair_start[ab], npab = PV.pair_start[ab + 1] - ab0;
  const int cd0 = PV.pair_start[cd], npcd = PV.pair_start[cd + 1] - cd0;
  const int np = npab * npcd;
  const double pi52 = 17.493418327624862846;  // pi^{5/2}
  double O[NE];
#pragma unroll
  for (int i = 0; i < NE; ++i) O[i] = 0.0;
  unsigned nproc = 0;
  for (int r = lane; r < np; r += 32) {
    const int iab = r / npcd, icd = r - iab * npcd;
    const int pab = ab0 + iab, pcd = cd0 + icd;
    const int64_t pq = QV.pq_off[q] + r - pq0;
    if (keys[pq * nf] == kSkipKey) continue;   // dropped by the primitive screen
    ++nproc;
    // g_n = sqrt(pi^5/(p+q))/(pq) * sum over families (fixed order)
    const double p = PV.pp_p[pab], qq = PV.pp_p[pcd];
    const double pref = pi52 / (sqrt(p + qq) * p * qq);
    double g[L + 1];
#pragma unroll
    for (int n = 0; n <= L; ++n) g[n] = 0.0;
    for (int f = 0; f < nf; ++f) {
      const double *pp = part + (pq * nf + f) * kPartPitch;
#pragma unroll
      for (int n = 0; n <= L; ++n) g[n] += pp[n];
    }
#pragma unroll
    for (int n = 0; n <= L; ++n) g[n] *= pref;
    const double X = pair_sep(PV.pp_P, pab, pcd, 0), Y = pair_sep(PV.pp_P, pab, pcd, 1),
                 Z = pair_sep(PV.pp_P, pab, pcd, 2);
    // Hermite recursion, levels n = L .. 0, in registers (every index is a
    // compile-time constant after unrolling)
    double R[NH], Rn[NH];
    R[0] = g[L];
#pragma unroll
    for (int n = L - 1; n >= 0; --n) {
#pragma unroll
      for (int S = 0; S <= L - n; ++S)
#pragma unroll
        for (int t = S; t >= 0; --t)
#pragma unroll
          for (int v = 0; v <= S - t; ++v) {
            const int u = S - t - v;
            double val;
            if (S == 0) val = g[n];
            else if (t > 0) val = X * R[hidx(t - 1, u, v)] + (t > 1 ? (t - 1) * R[hidx(t - 2, u, v)] : 0.0);
            else if (u > 0) val = Y * R[hidx(t, u - 1, v)] + (u > 1 ? (u - 1) * R[hidx(t, u - 2, v)] : 0.0);
            else val = Z * R[hidx(t, u, v - 1)] + (v > 1 ? (v - 1) * R[hidx(t, u, v - 2)] : 0.0);
            Rn[hidx(t, u, v)] = val;
          }
#pragma unroll
      for (int i = 0; i < NH; ++i) R[i] = Rn[i];
    }
    const double *Eab = PV.epool + PV.pp_eoff[pab];
    const double *Ecd = PV.epool + PV.pp_eoff[pcd];
    const double *Fab = Eab + 3 * N1AB;   // dE/dAB (I5)
    double c5 = 0.0;
    if constexpr (I5) {
      const double a = PV.pp_ab[2 * pab], b = PV.pp_ab[2 * pab + 1];
      c5 = (a - b) / (2.0 * (a + b));
    }
#pragma unroll
    for (int ic = 0; ic < NC; ++ic)
#pragma unroll
      for (int id = 0; id < ND; ++id) {
        const int cx = cart_i(LC, ic), cy = cart_j(LC, ic), cz = LC - cx - cy;
        const int dx = cart_i(LD, id), dy = cart_j(LD, id), dz = LD - dx - dy;
        const double *fx = Ecd + (cx * (LD + 1) + dx) * NTCD;
        const double *fy = Ecd + N1CD + (cy * (LD + 1) + dy) * NTCD;
        const double *fz = Ecd + 2 * N1CD + (cz * (LD + 1) + dz) * NTCD;
        // ket sums W(T,U,V) = sum E^{cd}_{t'u'v'} R_{T+t',U+u',V+v'} for every bra
        // Hermite index the block needs (T+U+V <= lab + EXT)
        constexpr int LBH = LA + LB + EXT;
        constexpr int NHB = (LBH + 1) * (LBH + 2) * (LBH + 3) / 6;
        double W[NHB];
#pragma unroll
        for (int S = 0; S <= LBH; ++S)
#pragma unroll
          for (int T = S; T >= 0; --T)
#pragma unroll
            for (int V = 0; V <= S - T; ++V) {
              const int U = S - T - V;
              double w = 0.0;
#pragma unroll
              for (int t2 = 0; t2 <= cx + dx; ++t2)
#pragma unroll
                for (int u2 = 0; u2 <= cy + dy; ++u2)
#pragma unroll
                  for (int v2 = 0; v2 <= cz + dz; ++v2)
                    if (T + t2 + U + u2 + V + v2 <= L) w = fma(fx[t2] * fy[u2] * fz[v2], R[hidx(T + t2, U + u2, V + v2)], w);
              W[hidx(T, U, V)] = w;
            }
#pragma unroll
        for (int ia = 0; ia < NA; ++ia)
#pragma unroll
          for (int ib = 0; ib < NB; ++ib) {
            const int ax = cart_i(LA, ia), ay = cart_j(LA, ia), az = LA - ax - ay;
            const int bx = cart_i(LB, ib), by = cart_j(LB, ib), bz = LB - bx - by;
            const int ox = (ax * (LB + 1) + bx) * NTAB, oy = N1AB + (ay * (LB + 1) + by) * NTAB,
                      oz = 2 * N1AB + (az * (LB + 1) + bz) * NTAB;
            double acc = 0.0;
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
              for (int u = 0; u <= ay + by; ++u)
#pragma unroll
                for (int v = 0; v <= az + bz; ++v) {
                  double term;
                  if constexpr (I5) {
                    const double lap = W[hidx(t + 2, u, v)] + W[hidx(t, u + 2, v)] + W[hidx(t, u, v + 2)];
                    term = c5 * Eab[ox + t] * Eab[oy + u] * Eab[oz + v] * lap;
                    term -= Fab[ox + t] * Eab[oy + u] * Eab[oz + v] * W[hidx(t + 1, u, v)];
                    term -= Eab[ox + t] * Fab[oy + u] * Eab[oz + v] * W[hidx(t, u + 1, v)];
                    term -= Eab[ox + t] * Eab[oy + u] * Fab[oz + v] * W[hidx(t, u, v + 1)];
                  } else {
                    term = Eab[ox + t] * Eab[oy + u] * Eab[oz + v] * W[hidx(t, u, v)];
                  }
                  acc += ((t + u + v) & 1) ? -term : term;
                }
            O[((ia * NB + ib) * NC + ic) * ND + id] += acc;
          }
      }
  }
  // the lanes' sums, by a fixed butterfly (every lane ends with the total)
#pragma unroll
  for (int i = 0; i < NE; ++i) {
    double v = O[i];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    O[i] = v;
  }
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NE; ++i) out_q[i] = O[i];
  }
  if (flops_total) {
    // the same algorithmic count per primitive quartet as the general kernel
    unsigned tot = nproc;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0 && tot) {
      const unsigned long long r = 2ull * (L + 1) * (L + 2) * (L + 3) * (L + 4) / 24;
      const unsigned long long ket = 2ull * nh_count(LA + LB + EXT) * nh_count(LC + LD) * (NC * ND);
      const unsigned long long bra = 2ull * (NA * NB) * nh_count(LA + LB) * (NC * ND) * (I5 ? 4 : 1);
      atomicAdd(flops_total, (unsigned long long)tot * (r + ket + bra));
    }
  }
}

// range == null: tasks [0, ntask), one warp each, pair data PV, blocks into
// out.  range != null (the batch engine's persistent launch): the tasks
// [range[0], range[1]) in grid-stride order, each quartet's pair data and
// output array from its request's slot.
template <int LA, int LB, int LC, int LD, bool I5>
__global__ void __launch_bounds__(32 * kThinWarps)
k_contract_thin(PairView PV, QuartetView QV, int nf, int64_t pq0, const CTask *tasks, int64_t ntask,
                const int64_t *range, const int *keys, const double *part, double *out, const int64_t *offsets,
                unsigned long long *flops_total) {
  const int64_t warp = (int64_t)blockIdx.x * kThinWarps + (threadIdx.x >> 5);
  if (!range) {
    if (warp >= ntask) return;   // warp-uniform
    const int64_t q = tasks[warp].q;
    thin_quartet_body<LA, LB, LC, LD, I5>(PV, QV, nf, pq0, q, keys, part, out + offsets[q], flops_total);
    return;
  }
  const int64_t t1 = range[1], stride = (int64_t)gridDim.x * kThinWarps;
  for (int64_t tk = range[0] + warp; tk < t1; tk += stride) {
    const int64_t q = tasks[tk].q;
    const int slot = QV.qslot[q];
    thin_quartet_body<LA, LB, LC, LD, I5>(QV.slot_view[slot], QV, nf, pq0, q, keys, part,
                                          QV.slot_out[slot] + offsets[q], flops_total);
  }
}

// Class keys (la << 6 | lb << 4 | lc << 2 | ld): every (la, lb, lc, ld) with
// la + lb + lc + ld <= 2 (in two groups), and with la + lb + lc + ld = 3 (in
// four): the instances are compiled in seven parts, in parallel.
#define F12_THIN_KEYS_2A(X) X(0x00) X(0x01) X(0x04) X(0x10) X(0x40) X(0x02) X(0x08) X(0x20)
#define F12_THIN_KEYS_2B(X) X(0x80) X(0x05) X(0x11) X(0x41) X(0x14) X(0x44) X(0x50)
#define F12_THIN_KEYS_2(X) F12_THIN_KEYS_2A(X) F12_THIN_KEYS_2B(X)
#define F12_THIN_KEYS_3A(X) X(0x03) X(0x0C) X(0x30) X(0xC0) X(0x06)
#define F12_THIN_KEYS_3B(X) X(0x09) X(0x12) X(0x18) X(0x21) X(0x24)
#define F12_THIN_KEYS_3C(X) X(0x42) X(0x48) X(0x60) X(0x81) X(0x84)
#define F12_THIN_KEYS_3D(X) X(0x90) X(0x15) X(0x45) X(0x51) X(0x54)
#define F12_THIN_KEYS_3(X) F12_THIN_KEYS_3A(X) F12_THIN_KEYS_3B(X) F12_THIN_KEYS_3C(X) F12_THIN_KEYS_3D(X)

template <int K, bool I5>
ThinKernel thin_entry() {
  return &k_contract_thin<(K >> 6) & 3, (K >> 4) & 3, (K >> 2) & 3, K & 3, I5>;
}

// Part p (thin_inst.cu compiled with F12_THIN_PART = p) of the instances: the
// kernel for (key, i5) if the part holds it, else null.
ThinKernel thin_part0(int key, bool i5);   // L <= 2, not I5
ThinKernel thin_part1(int key, bool i5);   // L = 3, not I5 (four parts)
ThinKernel thin_part2(int key, bool i5);
ThinKernel thin_part3(int key, bool i5);
ThinKernel thin_part4(int key, bool i5);
ThinKernel thin_part5(int key, bool i5);   // I5, L <= 2 (two parts)
ThinKernel thin_part6(int key, bool i5);

}  // namespace f12k
