// Double-float (hi + lo, two floats, 48-bit significand) kernels for the R x R
// normal-equation work of the FP32 and MIXED_BF16 modes (Sec. 2.3; the
// normal-equation steps of Algorithms 1 and 3).
//
// GB300's float64 pipe runs at 1/64 of the float32 rate, costs a full warp
// cycle even for partially active warps and takes ~1,100 cycles for a
// reciprocal square root, so the Gram matrices, the Cholesky factorisation of
// Gamma and the row solves run here in double-float arithmetic on the float32
// pipes.  The building blocks are the classical error-free transformations:
// TwoSum (Knuth), FastTwoSum (Dekker), TwoProd via FMA, and the double-word
// addition/multiplication built from them (accurate variants, relative error
// a few units of 2^-48).  Rounding-sensitive steps use __f*_rn intrinsics so
// the compiler cannot contract or reassociate them.  The float64 mode keeps
// the IEEE float64 kernels of small.cu.
#include <algorithm>

#include <cooperative_groups.h>

#include "dfloat.cuh"
#include "internal.h"
#include "jacobi.cuh"

namespace cg = cooperative_groups;

namespace cpals {

namespace {

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

using namespace dfa;

// ---------------------------------------------------------------- split
__global__ void split_kernel(const double* __restrict__ A, float* __restrict__ hi,
                             float* __restrict__ lo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const dfl d = df_of(A[i]);
    hi[i] = d.hi;
    lo[i] = d.lo;
  }
}

// ---------------------------------------------------------------- Grams
// S = A^T A with A = Ahi + Alo: every product's leading part is exact
// (TwoProd), sums are compensated (TwoSum, the Dot2 scheme of Ogita, Rump and
// Oishi) and the cross terms hi*lo are added in float: the tile comes out as
// if accumulated in twice the float precision.  W = Aw^T dAw (float; only the
// second-order PP terms use it).  One thread-block cluster per 32 x 32 output
// tile; its CTAs take consecutive row chunks, keep their partial tile in
// shared memory and, after a cluster barrier, each CTA adds one slice of the
// tile over all partials (distributed shared memory, split order) and writes
// it: no global partials, fences or atomics.  CTA 0 of the grid also sums
// the per-row ||dA||^2 and ||A||^2 of the row solve (written by the previous
// kernel) in a fixed order.
__global__ void __launch_bounds__(256)
gram_df_kernel(const float* __restrict__ Ahi, const float* __restrict__ Alo,
               const float* __restrict__ Aw, const float* __restrict__ dAw, int s, int R, int nb,
               int ntS, int splits, int chunk, double* __restrict__ S, float* __restrict__ Shi,
               float* __restrict__ Slo, float* __restrict__ W, const float2* __restrict__ rownorm,
               double* __restrict__ scal, const float* __restrict__ ShiAll,
               const float* __restrict__ SloAll, int N, int n, int nn, float2* __restrict__ Gpk) {
  cg::cluster_group cl = cg::this_cluster();
  const int z = (int)cl.block_rank();
  const int t = blockIdx.x / splits;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int y0 = z * chunk, y1 = min(s, y0 + chunk);
  __shared__ float Ah[32][33], Al[32][33], Bh[32][33], Bl[32][33];
  __shared__ float2 part[1024];
  int ti, tj;
  if (t < ntS) {
    int tt = t;
    ti = 0;
    while (tt >= nb - ti) { tt -= nb - ti; ti++; }
    tj = ti + tt;
    float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
    for (int yb = y0; yb < y1; yb += 32) {
      for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
        const int yy = idx / 32, c = idx % 32;
        const int y = yb + yy;
        const int ci = ti * 32 + c, cj = tj * 32 + c;
        const bool vi = y < y1 && ci < R, vj = y < y1 && cj < R;
        Ah[yy][c] = vi ? Ahi[(int64_t)y * R + ci] : 0.f;
        Al[yy][c] = vi ? Alo[(int64_t)y * R + ci] : 0.f;
        Bh[yy][c] = vj ? Ahi[(int64_t)y * R + cj] : 0.f;
        Bl[yy][c] = vj ? Alo[(int64_t)y * R + cj] : 0.f;
      }
      __syncthreads();
#pragma unroll 4
      for (int yy = 0; yy < 32; yy++) {
        const float bh = Bh[yy][tx], bl = Bl[yy][tx];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const float ah = Ah[yy][ty + 8 * q], al = Al[yy][ty + 8 * q];
          const dfl pr = two_prod(ah, bh);
          const dfl su = two_sum(sh[q], pr.hi);
          sh[q] = su.hi;
          sl[q] = __fadd_rn(sl[q], __fadd_rn(su.lo, __fadd_rn(pr.lo, __fmaf_rn(ah, bl, __fmul_rn(al, bh)))));
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; q++) part[(ty + 8 * q) * 32 + tx] = pk(fast_two_sum(sh[q], sl[q]));
  } else {
    ti = (t - ntS) / nb;
    tj = (t - ntS) % nb;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int yb = y0; yb < y1; yb += 32) {
      for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
        const int yy = idx / 32, c = idx % 32;
        const int y = yb + yy;
        const int ci = ti * 32 + c, cj = tj * 32 + c;
        Ah[yy][c] = (y < y1 && ci < R) ? Aw[(int64_t)y * R + ci] : 0.f;
        Bh[yy][c] = (y < y1 && cj < R) ? dAw[(int64_t)y * R + cj] : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int yy = 0; yy < 32; yy++) {
        const float bj = Bh[yy][tx];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[q] = fmaf(Ah[yy][ty + 8 * q], bj, acc[q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; q++) part[(ty + 8 * q) * 32 + tx] = make_float2(acc[q], 0.f);
  }
  cl.sync();                                   // every partial tile is in its CTA's shared memory
  // this CTA's slice of the tile, summed over the partials in split order
  const int per = (1024 + splits - 1) / splits;
  const int eend = min(1024, z * per + per);
  for (int e = z * per + (int)threadIdx.x; e < eend; e += blockDim.x) {
    float2 v[8];
#pragma unroll
    for (int zz = 0; zz < 8; zz++)
      if (zz < splits) v[zz] = *cl.map_shared_rank(&part[e], zz);
    dfl acc = upk(v[0]);
#pragma unroll
    for (int zz = 1; zz < 8; zz++)
      if (zz < splits) acc = t < ntS ? df_add(acc, upk(v[zz])) : dfl{acc.hi + v[zz].x, 0.f};
    const int i = ti * 32 + e / 32, j = tj * 32 + e % 32;
    // a diagonal tile holds both (i, j) and (j, i), summed in different
    // orders: only i <= j writes the pair, so S is exactly symmetric and
    // every run writes the same value
    if (i < R && j < R && !(t < ntS && ti == tj && i > j)) {
      if (t < ntS) {
        const double d = df_dbl(acc);
        S[i * R + j] = d;
        S[j * R + i] = d;
        Shi[i * R + j] = acc.hi;
        Shi[j * R + i] = acc.hi;
        Slo[i * R + j] = acc.lo;
        Slo[j * R + i] = acc.lo;
        if (Gpk && i <= j) {
          // Gamma^(nn)_ji = product over k != nn of S^(k)_ij, in mode order,
          // packed by columns (entry (j, i), j >= i, at cs(i) + j - i)
          dfl g = {1.f, 0.f};
          const int RR = R * R;
          for (int k = 0; k < N; k++) {
            if (k == nn) continue;
            const dfl sk = k == n ? acc : dfl{ShiAll[(int64_t)k * RR + i * R + j],
                                              SloAll[(int64_t)k * RR + i * R + j]};
            g = df_mul(g, sk);
          }
          Gpk[i * R - i * (i - 1) / 2 + (j - i)] = pk(g);
        }
      } else {
        W[i * R + j] = acc.hi;
      }
    }
  }
  cl.sync();                                   // no CTA leaves while its partial is being read
  if (blockIdx.x != 0) return;
  // per-row ||dA||^2 and ||A||^2 (double-float) reduced in a fixed order
  __shared__ float2 rd[256], ra[256];
  dfl a = {0.f, 0.f}, b = {0.f, 0.f};
  for (int y = threadIdx.x; y < s; y += blockDim.x) {
    a = df_add(a, upk(rownorm[2 * y]));
    b = df_add(b, upk(rownorm[2 * y + 1]));
  }
  rd[threadIdx.x] = pk(a);
  ra[threadIdx.x] = pk(b);
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      rd[threadIdx.x] = pk(df_add(upk(rd[threadIdx.x]), upk(rd[threadIdx.x + st])));
      ra[threadIdx.x] = pk(df_add(upk(ra[threadIdx.x]), upk(ra[threadIdx.x + st])));
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scal[0] = df_dbl(upk(rd[0]));
    scal[1] = df_dbl(upk(ra[0]));
  }
}

// ---------------------------------------------------------------- Gamma, Cholesky, inverse
// A cluster of five CTAs forms Gamma^(n) = Hadamard product of the Grams
// S^(k), k != n, in double-float, factors it Gamma = L L^T and inverts the
// factor, W = L^-1, two pivots (one column pair P = (p, p+1), p = 2P) per
// step (right-looking; Golub & Van Loan Alg. 4.2.2 for the factor, the
// column-oriented triangular inverse for W).
//   CTA 0 (chain) makes the pairs.  Its pivot warp factors the 2 x 2 pivot
//     block (a, b; b, d) of pair P as il2 = 1/sqrt(a), il3 = a il2 /
//     sqrt(ad - b^2) (two independent reciprocal square roots) and then forms
//     rows p+2 and p+3 of the pair itself, so the next pivot block never
//     waits for another warp.  Row thread i forms L_ip and L_i,p+1 and the
//     inverse-update coefficients v_i = L_i,p+1 / L_p+1,p+1, u_i = L_ip / L_pp
//     - v_i L_p+1,p / L_pp.
//   CTAs 2 and 4 (trailing updates) hold the lower triangle of Gamma for the
//     column pairs of their parity (pairs Q with Q % 2 = 0 on CTA 2, odd on
//     CTA 4), packed by columns.  For each pair P they apply P to their
//     columns of pairs >= P+3; the owner of pair P+3 does those columns first
//     and sends them to CTA 0.  A column pair thus reaches CTA 0 three pairs
//     ahead, with every pair up to Q-3 applied; CTA 0 applies pairs Q-2 and
//     Q-1 (in that order) itself, so its chain never waits for a trailing
//     update and the two halves of the trailing work run side by side.
//   CTAs 1 and 3 (inverse) hold the columns of the inverse in progress of
//     their parity (even columns on CTA 1, odd on CTA 3; row i at ro[i]),
//     initially the identity, and apply B_ic -= u_i B_kc + v_i B_k+1,c for
//     rows i >= k+2, columns c <= k+1 per pair k = 2P (pivot k and pivot k+1,
//     which sees row k+1 after pivot k).  Row k+1 gets pivot k at the end,
//     and row j of W is the final row j of B divided by L_jj.
// Data moves between the CTAs only as st.async stores into the receiver's
// shared memory that complete a transaction count on one of its mbarriers
// (one per pair and purpose), so no CTA reads another's shared memory and
// no fence is needed; every wait is bounded.  Every update is one fused
// double-float g - a b - c d (exact leading products and sums, one
// renormalisation: backward error a few units of 2^-48 relative to the
// operands).  Writes W (row stride RS = R | 1, zeros above the diagonal and
// in the padding column) and, with useV, the float matrix Z of the
// second-order PP terms (Eq. 3).  A non-positive pivot sets bit n of
// status[0]; a wait that runs out sets a bit of status[2].
#ifndef CPALS_CHOL_THREADS
#define CPALS_CHOL_THREADS 512
#endif
constexpr int kLook = 3;        // pairs a column pair travels ahead of its use
__host__ __device__ __forceinline__ int col_start(int j, int R) { return j * R - j * (j - 1) / 2; }
// g - a b - c d
__device__ __forceinline__ dfl df_fms2(dfl g, dfl a, dfl b, dfl c, dfl d) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  e1 = __fmaf_rn(a.hi, b.lo, e1);
  e1 = __fmaf_rn(a.lo, b.hi, e1);
  const float p2 = __fmul_rn(c.hi, d.hi);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  e2 = __fmaf_rn(c.hi, d.lo, e2);
  e2 = __fmaf_rn(c.lo, d.hi, e2);
  const dfl s = two_sum(g.hi, -p1);
  const dfl t = two_sum(s.hi, -p2);
  const float lo = __fsub_rn(__fsub_rn(__fadd_rn(__fadd_rn(g.lo, s.lo), t.lo), e1), e2);
  return fast_two_sum(t.hi, lo);
}
__device__ __forceinline__ dfl df_fms(dfl g, dfl a, dfl b) {   // g - a b
  return df_add_fast(g, df_neg(df_mul(a, b)));
}
__device__ __forceinline__ bool bad_pivot(dfl p) { return !(p.hi > 0.f) || !isfinite(p.hi); }
__device__ __forceinline__ dfl lo2(float4 v) { return {v.x, v.y}; }
__device__ __forceinline__ dfl hi2(float4 v) { return {v.z, v.w}; }
__device__ __forceinline__ float4 pk2(dfl a, dfl b) { return make_float4(a.hi, a.lo, b.hi, b.lo); }
// g - (pair P-2 terms) - (pair P-1 terms): u2, v2 and u1, v1 hold the two
// rows' (L_.,q, L_.,q+1) of those pairs.  Four exact leading products, one
// chain of TwoSums on the high words, one renormalisation.
__device__ __forceinline__ dfl df_fms4(dfl g, float4 u2, float4 v2, float4 u1, float4 v1) {
  const dfl a[4] = {lo2(u2), hi2(u2), lo2(u1), hi2(u1)};
  const dfl b[4] = {lo2(v2), hi2(v2), lo2(v1), hi2(v1)};
  float p[4], e[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    p[k] = __fmul_rn(a[k].hi, b[k].hi);
    e[k] = __fmaf_rn(a[k].hi, b[k].hi, -p[k]);
    e[k] = __fmaf_rn(a[k].hi, b[k].lo, e[k]);
    e[k] = __fmaf_rn(a[k].lo, b[k].hi, e[k]);
  }
  dfl s = two_sum(g.hi, -p[0]);
  float lo = __fadd_rn(g.lo, s.lo);
#pragma unroll
  for (int k = 1; k < 4; k++) {
    s = two_sum(s.hi, -p[k]);
    lo = __fadd_rn(lo, s.lo);
  }
  lo = __fsub_rn(__fsub_rn(lo, __fadd_rn(e[0], e[1])), __fadd_rn(e[2], e[3]));
  return fast_two_sum(s.hi, lo);
}

// Entries of the inverse held by the CTA of column parity h: row i keeps
// columns c <= i with c % 2 == h, at ro(i) + c / 2.
__host__ __device__ __forceinline__ int inv_tri(int x) { return x >= 1 ? ((x - 1) / 2) * (x / 2) : 0; }
__host__ __device__ __forceinline__ int inv_ro(int i, int h) {
  return h ? (i >= 1 ? (i - 1) + inv_tri(i - 1) : 0) : i + inv_tri(i);
}
// Packed entries of column pair Q (columns 2Q, 2Q+1, rows from the column down).
__host__ __device__ __forceinline__ int pair_cnt(int Q, int R) {
  const int p = 2 * Q;
  return (R - p) + (p + 1 < R ? R - p - 1 : 0);
}

// Shared-memory layout (byte offsets from the dynamic base).  Arrays that
// receive remote stores sit at the same offset in every CTA.
struct CholLayout {
  size_t gc, lc, end0;                        // CTA 0: pair columns (4 slots), L pairs (8 sets)
  size_t B, ro, uv, id, lsub, bars, flag, end1;   // inverse CTAs
  size_t G, crd, lcs, lc2, end2;              // trailing CTAs
  __host__ __device__ CholLayout(int R) {
    const int npair = (R + 1) / 2;
    auto al = [](size_t x) { return (x + 15) / 16 * 16; };
    gc = 0;
    lc = gc + al(4 * 2 * (size_t)R * 8);
    end0 = lc + 8 * (size_t)R * 16;
    B = 0;
    ro = al((size_t)inv_ro(R, 0) * 8);
    uv = ro + al((size_t)R * 4);
    id = uv + (size_t)npair * R * 16;
    lsub = id + al((size_t)R * 8);
    bars = lsub + al((size_t)R * 8);
    flag = bars + (size_t)npair * 8;
    end1 = flag + 16;
    int gmax = 0;
    for (int h = 0; h < 2; h++) {
      int c = 0;
      for (int Q = h; Q < npair; Q += 2) c += pair_cnt(Q, R);
      gmax = c > gmax ? c : gmax;
    }
    G = 0;
    crd = al((size_t)gmax * 8);
    lcs = crd + al((size_t)gmax * 4);
    lc2 = lcs + al((size_t)(npair / 2 + 2) * 4);
    end2 = lc2 + 8 * (size_t)R * 16;
  }
  __host__ __device__ size_t bytes() const {
    const size_t m = end0 > end1 ? end0 : end1;
    return m > end2 ? m : end2;
  }
};

// Remote shared-memory stores that complete a transaction count on an
// mbarrier of the receiving CTA (no fence on the sending side).
__device__ __forceinline__ uint32_t cluster_addr(const void* local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async16(uint32_t dst, float4 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
               ::"r"(dst), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar) : "memory");
}
__device__ __forceinline__ void st_async8(uint32_t dst, float2 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
               ::"r"(dst), "f"(v.x), "f"(v.y), "r"(bar) : "memory");
}
__device__ __forceinline__ void st_release_cluster(int* p, int v) {
  asm volatile("st.release.cluster.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_cluster(const int* p) {
  int v;
  asm volatile("ld.acquire.cluster.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __cluster_dims__(5, 1, 1) __launch_bounds__(CPALS_CHOL_THREADS, 1)
chol_inv_df_kernel(const float* __restrict__ Shi, const float* __restrict__ Slo,
                   const float* __restrict__ Wg, const float2* __restrict__ Gpk, int N, int n,
                   int R, float2* __restrict__ Wout, float* __restrict__ Z, int useV,
                   int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char csm[];
  __shared__ int bad;
  // CTA 0: mbX[P] (pair P's columns are here), mbR[P] (rows p, p+1 hold pair
  // P-1), mbR2[P] (rows p+2, p+3 hold pair P-1), mbC[P] (pair P's pivot block
  // is published); trailing CTAs: mbY[P] (every row of pair P is here)
  __shared__ __align__(8) uint64_t mbX[kMaxRank / 2], mbR[kMaxRank / 2], mbR2[kMaxRank / 2],
      mbC[kMaxRank / 2], mbY[kMaxRank / 2];
  __shared__ float2 piv[4][4];                 // per pair slot: il2, il3, c3 = L_p+1,p, c3 il2
  cg::cluster_group cl = cg::this_cluster();
  const int role = (int)cl.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  const int RR = R * R;
  const int RS = R | 1;
  const CholLayout lay(R);
  const int npair = (R + 1) / 2;
  float2* gc = reinterpret_cast<float2*>(csm + lay.gc);           // [slot][column of the pair][row]
  float4* lc = reinterpret_cast<float4*>(csm + lay.lc);           // [set][row] (L_ip, L_i,p+1)
  float2* B = reinterpret_cast<float2*>(csm + lay.B);
  int* ro = reinterpret_cast<int*>(csm + lay.ro);
  float4* UV = reinterpret_cast<float4*>(csm + lay.uv);
  float2* id = reinterpret_cast<float2*>(csm + lay.id);
  float2* lsub = reinterpret_cast<float2*>(csm + lay.lsub);
  uint64_t* bars = reinterpret_cast<uint64_t*>(csm + lay.bars);   // one per pair of columns
  int* flag = reinterpret_cast<int*>(csm + lay.flag);             // [0] stop
  float2* G = reinterpret_cast<float2*>(csm + lay.G);
  uint32_t* crd = reinterpret_cast<uint32_t*>(csm + lay.crd);
  int* lcs = reinterpret_cast<int*>(csm + lay.lcs);               // local start of owned pairs
  float4* lc2 = reinterpret_cast<float4*>(csm + lay.lc2);
  auto mb_init = [](uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(count));
  };
  auto mb_expect = [](uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(bytes) : "memory");
  };
  // hint: suspend-time hint in ns (0: poll); a waiting thread sleeps until the
  // phase completes instead of spinning on the pipe the pivot warp uses
  auto mwait = [&](uint64_t* bar, int code, uint32_t hint = 0) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    {
      uint32_t done;   // fast path: already complete, no clock read
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
                   " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(b) : "memory");
      if (done) return;
    }
    const unsigned long long t0 = clock64();
    while (true) {
      uint32_t done;
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0, %2;\n"
                   " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(b), "r"(hint) : "memory");
      if (done) return;
      if (clock64() - t0 > 4000000000ull) {
        atomicOr(status + 2, code);
        bad = 1;
        return;
      }
    }
  };
  // barriers completed by this CTA's own threads need only CTA-scope acquire
  auto mwait_cta = [&](uint64_t* bar, int code, uint32_t hint = 0) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    {
      uint32_t done;
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                   " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(b) : "memory");
      if (done) return;
    }
    const unsigned long long t0 = clock64();
    while (true) {
      uint32_t done;
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, %2;\n"
                   " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(b), "r"(hint) : "memory");
      if (done) return;
      if (clock64() - t0 > 4000000000ull) {
        atomicOr(status + 2, code);
        bad = 1;
        return;
      }
    }
  };
  auto marrive = [](uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
  };
  const bool inv = role == 1 || role == 3, trl = role == 2 || role == 4;
  const int par = inv ? (role - 1) / 2 : trl ? (role - 2) / 2 : 0;   // column (pair) parity
  if (tid == 0) bad = 0;
  if (role == 0) {
    for (int P = tid; P < npair; P += nt) {
      mb_init(mbX + P, 1);
      if (P >= kLook) mb_expect(mbX + P, 8u * (uint32_t)pair_cnt(P, R));   // the first ones: formed here
      mb_init(mbR + P, min(2, R - 2 * P));
      mb_init(mbR2 + P, max(1, min(2, R - 2 * P - 2)));   // waited only when the rows exist
      mb_init(mbC + P, 1);
    }
  } else if (trl) {
    for (int P = tid; P < npair; P += nt) {
      mb_init(mbY + P, 1);
      mb_expect(mbY + P, 16u * (uint32_t)(R - 2 * P));
    }
    if (tid == 0) {
      int c = 0;
      for (int Q = par, k = 0; Q < npair; Q += 2, k++) {
        lcs[k] = c;
        c += pair_cnt(Q, R);
      }
      lcs[(npair - par + 1) / 2] = c;                // end of the owned entries
    }
  } else {
    if (tid == 0) flag[0] = 0;
    // pair P brings 16 bytes per row i >= 2P, 1/L_jj of its columns and,
    // when it has two, L_{2P+1,2P} / L_{2P,2P}
    for (int P = tid; P < npair; P += nt) {
      const uint32_t b = (uint32_t)__cvta_generic_to_shared(bars + P);
      const uint32_t bytes = 16u * (uint32_t)(R - 2 * P) + (2 * P + 1 < R ? 24u : 8u);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
                   : "memory");
    }
    for (int i = tid; i < R; i += nt) ro[i] = inv_ro(i, par);
    // identity (columns of this parity)
    for (int i = warp; i < R; i += nwarp) {
      const int o = inv_ro(i, par);
      for (int c = 2 * lane + par; c <= i; c += 64) B[o + (c >> 1)] = make_float2(c == i ? 1.f : 0.f, 0.f);
    }
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  cl.sync();                                   // every CTA's barriers exist before anyone sends
  if (trl) {
    // ---------------------------------------------------------- trailing updates
    const uint32_t gcr = cluster_addr(gc, 0), mbXr = cluster_addr(mbX, 0);
    const int nown = (npair - par + 1) / 2;
    const int gtot = lcs[nown];
    // (row, column) of every owned entry, and Gamma there
    for (int e = tid; e < gtot; e += nt) {
      int k = 0;
      while (k + 1 < nown && lcs[k + 1] <= e) k++;
      const int Q = par + 2 * k, p = 2 * Q;
      const int r = e - lcs[k];
      const int j = r < R - p ? p : p + 1;
      const int i = j == p ? p + r : p + 1 + (r - (R - p));
      crd[e] = (uint32_t)i | ((uint32_t)j << 16);
      dfl g = {1.f, 0.f};
      if (Gpk) {
        g = upk(Gpk[col_start(j, R) + i - j]);
      } else {
        for (int k2 = 0; k2 < N; k2++)
          if (k2 != n) g = df_mul(g, dfl{Shi[(int64_t)k2 * RR + i * R + j], Slo[(int64_t)k2 * RR + i * R + j]});
      }
      G[e] = pk(g);
    }
    __syncthreads();
    for (int P = 0; P < npair; P++) {
      if (tid == 0) mwait(mbY + P, 16, 2000);
      __syncthreads();                         // pair P is here; the previous updates are done
      const float4* cc = lc2 + (P & 7) * R;
      // G_ij -= L_i,p L_j,p + L_i,p+1 L_j,p+1 on [e0, e1), two entries per
      // iteration (independent double-float chains); out sends the result
      // to CTA 0's slot of pair Qs
      auto update = [&](int e0, int e1, int Qs) {
        int e = e0 + tid;
        for (; e + nt < e1; e += 2 * nt) {
          const uint32_t ij0 = crd[e], ij1 = crd[e + nt];
          const float4 li0 = cc[ij0 & 0xffffu], lj0 = cc[ij0 >> 16];
          const float4 li1 = cc[ij1 & 0xffffu], lj1 = cc[ij1 >> 16];
          const dfl g0 = df_fms2(upk(G[e]), lo2(li0), lo2(lj0), hi2(li0), hi2(lj0));
          const dfl g1 = df_fms2(upk(G[e + nt]), lo2(li1), lo2(lj1), hi2(li1), hi2(lj1));
          G[e] = pk(g0);
          G[e + nt] = pk(g1);
          if (Qs >= 0) {
            const int i0 = ij0 & 0xffffu, j0 = ij0 >> 16, i1 = ij1 & 0xffffu, j1 = ij1 >> 16;
            st_async8(gcr + 8u * (uint32_t)((((Qs & 3) * 2 + (j0 & 1)) * R) + i0), pk(g0), mbXr + 8u * (uint32_t)Qs);
            st_async8(gcr + 8u * (uint32_t)((((Qs & 3) * 2 + (j1 & 1)) * R) + i1), pk(g1), mbXr + 8u * (uint32_t)Qs);
          }
        }
        if (e < e1) {
          const uint32_t ij = crd[e];
          const float4 li = cc[ij & 0xffffu], lj = cc[ij >> 16];
          const dfl g = df_fms2(upk(G[e]), lo2(li), lo2(lj), hi2(li), hi2(lj));
          G[e] = pk(g);
          if (Qs >= 0)
            st_async8(gcr + 8u * (uint32_t)((((Qs & 3) * 2 + ((ij >> 16) & 1)) * R) + (ij & 0xffffu)), pk(g),
                      mbXr + 8u * (uint32_t)Qs);
        }
      };
      const int Qn = P + kLook;                // goes to CTA 0 once pair P is in
      if (Qn < npair && (Qn & 1) == par) update(lcs[(Qn - par) >> 1], lcs[((Qn - par) >> 1) + 1], Qn);
      int Qr = P + kLook + 1;                  // the rest: owned pairs >= P+4
      Qr += (Qr - par) & 1;
      if (Qr < npair) update(lcs[(Qr - par) >> 1], gtot, -1);
    }
  } else if (role == 0) {
    // ---------------------------------------------------------- chain
    uint32_t UVr[2], idr[2], lsubr[2], barr[2], lc2r[2], mbYr[2];
    for (int h = 0; h < 2; h++) {
      UVr[h] = cluster_addr(UV, 1 + 2 * h);
      idr[h] = cluster_addr(id, 1 + 2 * h);
      lsubr[h] = cluster_addr(lsub, 1 + 2 * h);
      barr[h] = cluster_addr(bars, 1 + 2 * h);
      lc2r[h] = cluster_addr(lc2, 2 + 2 * h);
      mbYr[h] = cluster_addr(mbY, 2 + 2 * h);
    }
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // the first kLook column pairs straight from Gamma (no pair applies to
    // them yet); same product order as the trailing CTAs and the Gram kernel
    const int cf = min(2 * kLook, R);
    for (int e = tid; e < col_start(cf, R); e += nt) {
      int j = 0;
      while (j + 1 < cf && col_start(j + 1, R) <= e) j++;
      const int i = j + e - col_start(j, R);
      dfl g = {1.f, 0.f};
      if (Gpk) {
        g = upk(Gpk[e]);
      } else {
        for (int k = 0; k < N; k++)
          if (k != n) g = df_mul(g, dfl{Shi[(int64_t)k * RR + i * R + j], Slo[(int64_t)k * RR + i * R + j]});
      }
      gc[(((j >> 1) & 3) * 2 + (j & 1)) * R + i] = pk(g);
    }
    __syncthreads();
    if (tid == 0)
      for (int P = 0; P < min(kLook, npair); P++) marrive(mbX + P);
    if (warp == 4) {
      // pivot warp.  It keeps rows p and p+1 of the two previous pairs in
      // registers (Lp1, Lq1: pair P-1; Lp2, Lq2: pair P-2; each (L_.,q,
      // L_.,q+1)) and, once it has published a pivot block, forms rows p+2
      // and p+3 of the pair itself (the row threads' operations in the same
      // order, so the values are identical).
      float4 Lp1 = z4, Lq1 = z4, Lp2 = z4, Lq2 = z4;
      for (int P = 0; P < npair; P++) {
        const int p = 2 * P;
        const bool two = p + 1 < R;
        const bool more = p + 2 < R;           // rows p+2 (and p+3) exist
        if (more && P >= 1) mwait_cta(mbR2 + P, 8);
        mwait(mbX + P, 8);
        const float2* g = gc + (P & 3) * 2 * R;
        // lane 0: a = G_pp, lane 1: b = G_p+1,p, lane 2: d = G_p+1,p+1;
        // lanes 3, 4: column p of rows p+2, p+3; lanes 5, 6: column p+1 of
        // rows p+2, p+3; each less pairs P-2 and P-1 (rows p+2, p+3 of those
        // pairs come from the row threads)
        const int ii = p + 2 + ((lane - 3) & 1);
        const bool rowl = lane >= 3 && lane < 7 && ii < R && two;
        float4 q1 = z4, q2 = z4;
        float2 gv = make_float2(0.f, 0.f);
        if (lane < 3) {
          gv = lane == 2 ? g[R + p + 1] : g[p + (lane == 1 ? 1 : 0)];
        } else if (rowl) {
          if (P >= 1) q1 = lc[((P - 1) & 7) * R + ii];
          if (P >= 2) q2 = lc[((P - 2) & 7) * R + ii];
          gv = lane < 5 ? g[ii] : g[R + ii];
        }
        dfl x = {1.f, 0.f};
        if (lane < (two ? 3 : 1) || rowl) {
          const float4 u1 = lane < 3 ? (lane >= 1 ? Lq1 : Lp1) : q1;
          const float4 u2 = lane < 3 ? (lane >= 1 ? Lq2 : Lp2) : q2;
          const bool vq = lane == 2 || lane >= 5;
          x = df_fms4(upk(gv), u2, vq ? Lq2 : Lp2, u1, vq ? Lq1 : Lp1);
        }
        const dfl a = {__shfl_sync(0xffffffffu, x.hi, 0), __shfl_sync(0xffffffffu, x.lo, 0)};
        const dfl bb = {__shfl_sync(0xffffffffu, x.hi, 1), __shfl_sync(0xffffffffu, x.lo, 1)};
        const dfl d = {__shfl_sync(0xffffffffu, x.hi, 2), __shfl_sync(0xffffffffu, x.lo, 2)};
        // lane 0: 1/sqrt(ad - b^2); lane 1: 1/sqrt(a)
        const dfl det = two ? df_fms(df_mul(a, d), bb, bb) : dfl{1.f, 0.f};
        const dfl rin = df_rsqrt(lane == 0 ? det : a);
        const dfl il2 = {__shfl_sync(0xffffffffu, rin.hi, 1), __shfl_sync(0xffffffffu, rin.lo, 1)};
        const dfl rdet = {__shfl_sync(0xffffffffu, rin.hi, 0), __shfl_sync(0xffffffffu, rin.lo, 0)};
        const dfl il3 = two ? df_mul(df_mul(rdet, a), il2) : dfl{0.f, 0.f};
        const dfl c3 = two ? df_mul(bb, il2) : dfl{0.f, 0.f};
        if (lane == 0) {
          if (bad_pivot(a) || bad_pivot(det)) bad = 1;
          piv[P & 3][0] = pk(il2);
          piv[P & 3][1] = pk(il3);
          piv[P & 3][2] = pk(c3);
          piv[P & 3][3] = pk(df_mul(c3, il2));
          marrive(mbC + P);
        }
        if (more) {
          // rows p+2 and p+3 of this pair: L_ip on lanes 3, 4, then L_i,p+1
          // on lanes 5, 6 (row threads' operations, same order)
          const dfl l2 = df_mul(x, il2);
          const int src = lane >= 5 ? lane - 2 : lane;
          const dfl l2s = {__shfl_sync(0xffffffffu, l2.hi, src), __shfl_sync(0xffffffffu, l2.lo, src)};
          const dfl l3 = two ? df_mul(df_fms(x, l2s, c3), il3) : dfl{0.f, 0.f};
          // the next pair's pivot rows p+2, p+3: this pair from l2, l3; pair
          // P-1 from what the row threads stored
          Lp2 = make_float4(__shfl_sync(0xffffffffu, q1.x, 3), __shfl_sync(0xffffffffu, q1.y, 3),
                            __shfl_sync(0xffffffffu, q1.z, 3), __shfl_sync(0xffffffffu, q1.w, 3));
          Lq2 = make_float4(__shfl_sync(0xffffffffu, q1.x, 4), __shfl_sync(0xffffffffu, q1.y, 4),
                            __shfl_sync(0xffffffffu, q1.z, 4), __shfl_sync(0xffffffffu, q1.w, 4));
          Lp1 = make_float4(__shfl_sync(0xffffffffu, l2.hi, 3), __shfl_sync(0xffffffffu, l2.lo, 3),
                            __shfl_sync(0xffffffffu, l3.hi, 5), __shfl_sync(0xffffffffu, l3.lo, 5));
          Lq1 = make_float4(__shfl_sync(0xffffffffu, l2.hi, 4), __shfl_sync(0xffffffffu, l2.lo, 4),
                            __shfl_sync(0xffffffffu, l3.hi, 6), __shfl_sync(0xffffffffu, l3.lo, 6));
        }
        __syncwarp();
      }
    } else if ((warp >= 1 && warp <= 3) || warp == 5) {
      // row threads (warps 1-3 and 5: the pivot warp, warp 4, has its
      // scheduler partition to itself, warps 0, 8 and 12 idle)
      const int i = warp == 5 ? 96 + lane : tid - 32;
      float4 q1 = z4, q2 = z4;                  // row i of pairs P-1 and P-2
      for (int P = 0; P < npair && 2 * P <= i && i < R; P++) {
        const int p = 2 * P;
        const bool two = p + 1 < R;
        if (P >= 1) mwait_cta(mbR + P, 8, 2000);
        mwait(mbX + P, 8, 2000);
        const float2* g = gc + (P & 3) * 2 * R;
        const float4 L1p = P >= 1 ? lc[((P - 1) & 7) * R + p] : z4;
        const float4 L1q = (two && P >= 1) ? lc[((P - 1) & 7) * R + p + 1] : z4;
        const float4 L2p = P >= 2 ? lc[((P - 2) & 7) * R + p] : z4;
        const float4 L2q = (two && P >= 2) ? lc[((P - 2) & 7) * R + p + 1] : z4;
        const dfl gi = df_fms4(upk(g[i]), q2, L2p, q1, L1p);
        dfl hi = {0.f, 0.f};
        if (two && i > p) hi = df_fms4(upk(g[R + i]), q2, L2q, q1, L1q);
        mwait_cta(mbC + P, 8, 2000);
        const dfl il2 = upk(piv[P & 3][0]), il3 = upk(piv[P & 3][1]);
        const dfl c3 = upk(piv[P & 3][2]), m = upk(piv[P & 3][3]);
        const dfl l2 = df_mul(gi, il2);
        const dfl l3 = (two && i > p) ? df_mul(df_fms(hi, l2, c3), il3) : dfl{0.f, 0.f};
        const float4 lv = pk2(l2, l3);
        lc[(P & 7) * R + i] = lv;
        if (P + 1 < npair && (i == p + 2 || i == p + 3)) marrive(mbR + P + 1);
        if (i == p + 4 || i == p + 5) marrive(mbR2 + P + 1);   // for the pivot warp
        for (int h = 0; h < 2; h++)
          st_async16(lc2r[h] + 16u * (uint32_t)((P & 7) * R + i), lv, mbYr[h] + 8u * (uint32_t)P);
        // inverse-update coefficients to both inverse CTAs
        const dfl q2v = df_mul(l2, il2);
        const dfl v = df_mul(l3, il3);
        const dfl u = df_fms(q2v, v, m);
        for (int h = 0; h < 2; h++) {
          const uint32_t bar = barr[h] + 8u * (uint32_t)P;
          st_async16(UVr[h] + 16u * (uint32_t)(P * R + i), pk2(u, v), bar);
          if (i == p) st_async8(idr[h] + 8u * p, pk(il2), bar);
          if (two && i == p + 1) {
            st_async8(idr[h] + 8u * (p + 1), pk(il3), bar);
            st_async8(lsubr[h] + 8u * (p + 1), pk(q2v), bar);
          }
        }
        q2 = q1;
        q1 = lv;
      }
    }
    __syncthreads();
    if (bad && tid == 0) {
      atomicOr(status, 1 << n);
      for (int h = 0; h < 2; h++) st_release_cluster(cl.map_shared_rank(flag, 1 + 2 * h), 1);   // stop the inverse CTAs
    }
  } else {
    // ---------------------------------------------------------- inverse (columns of parity par)
    if (useV) {
      // Z (second-order PP terms), entries split between the two inverse CTAs
      for (int idx = 2 * tid + par; idx < RR; idx += 2 * nt) {
        float zz = 0.f;
        for (int a = 0; a < N; a++) {
          if (a == n) continue;
          for (int b = a + 1; b < N; b++) {
            if (b == n) continue;
            float h = Wg[(int64_t)a * RR + idx] * Wg[(int64_t)b * RR + idx];
            for (int k = 0; k < N; k++)
              if (k != a && k != b && k != n) h *= Shi[(int64_t)k * RR + idx];
            zz += h;
          }
        }
        Z[idx] = zz;
      }
    }
    // thread 0 waits (bounded) for pair P or a stop; 0 = ready, 1 = stopped,
    // 2 = timed out; the caller's barrier publishes the state.  Two slots:
    // a wait writes the slot the other threads are not reading.
    __shared__ int state[2];
    int slot = 0;
    auto wait_pair = [&](int P, int sl) {
      if (tid == 0) {
        int st = 2;
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(bars + P);
        const unsigned long long t0 = clock64();
        while (clock64() - t0 < 4000000000ull) {
          uint32_t done;
          asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
                       " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(b) : "memory");
          if (done) { st = 0; break; }
          if (ld_acquire_cluster(flag)) { st = 1; break; }
        }
        state[sl] = st;
      }
    };
    // row i of W = (final row i of B) / L_ii; odd rows still lack pivot
    // i-1: B_i. -= (L_i,i-1 / L_i-1,i-1) B_i-1.  One warp per row, this
    // CTA's columns.
    auto write_row = [&](int i) {
      const dfl d = upk(id[i]);
      const bool odd = i & 1;
      const dfl f = odd ? upk(lsub[i]) : dfl{0.f, 0.f};
      const float2* Bi = B + ro[i];
      const float2* Bp = i >= 1 ? B + ro[i - 1] : B;
      for (int c = 2 * lane + par; c < RS; c += 64) {
        float2 w = make_float2(0.f, 0.f);
        if (c < i) {
          dfl b = upk(Bi[c >> 1]);
          if (odd) b = df_fms(b, f, upk(Bp[c >> 1]));
          w = pk(df_mul(b, d));
        } else if (c == i) {
          w = pk(d);
        }
        Wout[i * RS + c] = w;
      }
    };
    int st = 0;
    if (R > 2) wait_pair(0, 0);
    __syncthreads();
    for (int k = 0; k + 2 < R; k += 2) {
      st = state[slot];
      if (st) break;
      // (c) inverse update of rows >= k+2, this CTA's columns <= k+1
      const float4* cu = UV + (size_t)(k >> 1) * R;
      const int cols = (k + 2) >> 1, tot = (R - k - 2) * cols;
      if (tid < tot) {
        const float rc = 1.f / (float)cols;
        int q = (int)(((float)tid + 0.5f) * rc), c = tid - q * cols;
        const int dq = (int)(((float)nt + 0.5f) * rc), dc = nt - dq * cols;
        const float2* Bk = B + ro[k];
        const float2* Bk1 = B + ro[k + 1];
        const int ck = par ? (k >> 1) : (k >> 1) + 1;   // local columns <= k in row k
        // two entries per iteration (t and t + nt): independent chains
        int t = tid;
        for (; t + nt < tot; t += 2 * nt) {
          int q1 = q + dq, c1 = c + dc;
          if (c1 >= cols) {
            c1 -= cols;
            q1++;
          }
          const int i0 = k + 2 + q, i1 = k + 2 + q1;
          float2* bp0 = B + ro[i0] + c;
          float2* bp1 = B + ro[i1] + c1;
          const float4 w0 = cu[i0], w1 = cu[i1];
          const dfl bk0 = c < ck ? upk(Bk[c]) : dfl{0.f, 0.f};
          const dfl bk1 = c1 < ck ? upk(Bk[c1]) : dfl{0.f, 0.f};
          const dfl x0 = upk(*bp0), x1 = upk(*bp1);
          *bp0 = pk(df_fms2(x0, lo2(w0), bk0, hi2(w0), upk(Bk1[c])));
          *bp1 = pk(df_fms2(x1, lo2(w1), bk1, hi2(w1), upk(Bk1[c1])));
          q = q1 + dq;
          c = c1 + dc;
          if (c >= cols) {
            c -= cols;
            q++;
          }
        }
        if (t < tot) {
          const int i = k + 2 + q;
          float2* bp = B + ro[i] + c;
          const float4 w = cu[i];
          const dfl bk = c < ck ? upk(Bk[c]) : dfl{0.f, 0.f};
          *bp = pk(df_fms2(upk(*bp), lo2(w), bk, hi2(w), upk(Bk1[c])));
        }
      }
      // the next pair (or, after the last step, the last one for 1 / L_jj)
      slot ^= 1;
      wait_pair(k + 4 < R ? (k + 2) >> 1 : npair - 1, slot);
      __syncthreads();
    }
    if (R <= 2) {
      wait_pair(npair - 1, slot);
      __syncthreads();
    }
    if (!st) st = state[slot];
    if (st == 2 && tid == 0) atomicOr(status + 2, 2);
    if (!st)
      for (int i = warp; i < R; i += nwarp) write_row(i);
    if (st == 1 && tid == 0) {
      // stopped after a bad pivot: CTA 0 still sends every pair, so let them
      // all land (bounded) before this CTA may exit
      const unsigned long long t0 = clock64();
      for (int P = 0; P < npair; P++) {
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(bars + P);
        while (clock64() - t0 < 4000000000ull) {
          uint32_t done;
          asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
                       " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(b) : "memory");
          if (done) break;
        }
      }
    }
  }
  // no CTA exits while another may still store into its shared memory (every
  // expected store was waited for on an mbarrier, so no ordering is needed)
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

size_t chol_inv_smem(int R) { return CholLayout(R).bytes(); }

// ---------------------------------------------------------------- row solves
// Compensated dot-product accumulator (Dot2 of Ogita, Rump and Oishi, with
// the double-float operands' cross terms added to the compensation):
// s.hi is the running float sum, s.lo collects every rounding error.
__device__ __forceinline__ void dot2_acc(dfl& s, dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dfl t = two_sum(s.hi, p);
  s.hi = t.hi;
  s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, e));
}

// ---------------------------------------------------------------- Gamma^dagger
// Algorithm 1 writes the pseudo-inverse Gamma^dagger (Sec. 2.3).  When the
// factorisation above met a pivot that is not positive (status bit n), this
// CTA takes Gamma in float64 (from Gpk, else the Grams' hi + lo), finds
// Gamma = V diag(w) V^T by cyclic Jacobi and writes the factor
// W = diag(w^+)^(1/2) V^T in place of L^-1 (dense, row stride R|1), so that
// the row solve's a = W^T W b is b Gamma^dagger; eigenvalues at or below
// 1e-13 of the largest are dropped.  Status: bit n cleared and bit 16 + n
// set (the solve then runs over the dense W); a non-finite Gamma keeps bit n
// (an error).  Without a failed pivot the CTA only clears bit 16 + n.  V is
// accumulated in Wout's storage (R x R float64 fits in R x (R|1) float2).
__global__ void __launch_bounds__(512)
pinv_df_kernel(const float* __restrict__ Shi, const float* __restrict__ Slo,
               const float2* __restrict__ Gpk, int N, int n, int R, float2* __restrict__ Wout,
               int* __restrict__ status) {
  extern __shared__ double Gd[];
  __shared__ double w[kMaxRank];
  const int st = *reinterpret_cast<volatile int*>(status);
  const int tid = threadIdx.x, nt = blockDim.x;
  if (!((st >> n) & 1)) {
    if (tid == 0 && ((st >> (16 + n)) & 1)) atomicAnd(status, ~(1 << (16 + n)));
    return;
  }
  const int RR = R * R, RS = R | 1;
  double* V = reinterpret_cast<double*>(Wout);
  int fin = 1;
  for (int idx = tid; idx < RR; idx += nt) {
    const int i = idx / R, j = idx % R;
    double g = 1.0;
    if (Gpk) {
      const int a = max(i, j), b = min(i, j);
      const float2 v = Gpk[col_start(b, R) + a - b];
      g = (double)v.x + (double)v.y;
    } else {
      for (int k = 0; k < N; k++)
        if (k != n) g *= (double)Shi[(int64_t)k * RR + idx] + (double)Slo[(int64_t)k * RR + idx];
    }
    Gd[i * RS + j] = g;
    V[idx] = i == j ? 1.0 : 0.0;
    fin &= isfinite(g) ? 1 : 0;
  }
  if (!__syncthreads_and(fin)) return;
  sym_eig_jacobi(Gd, RS, V, R, R);
  pinv_weights(Gd, RS, R, true, w);
  for (int idx = tid; idx < RR; idx += nt) {
    const int k = idx / R, c = idx % R;
    Gd[k * RS + c] = w[k] * V[c * R + k];
  }
  __syncthreads();                             // every read of V precedes the first write of W
  for (int idx = tid; idx < RR; idx += nt) {
    const int k = idx / R, c = idx % R;
    Wout[k * RS + c] = pk(df_of(Gd[k * RS + c]));
  }
  if (tid == 0) {
    atomicAnd(status, ~(1 << n));
    atomicOr(status, 1 << (16 + n));
  }
}

// Row y of the normal equations, a Gamma = b (b = rhs, plus A_old Z for the
// second-order PP terms), solved as a = W^T (W b) with W = L^-1 from the
// factorisation kernel: two triangular products instead of two substitution
// chains, so every output entry is an independent compensated dot product.
// One CTA takes kRB rows at a time.  Two thread groups of Rp = R rounded up
// to 32 threads share the work: thread (h, r) sums half h of the terms of
// entry r (columns below / from the split point m), the halves are added in
// shared memory; W's zero triangle makes the loop bounds warp-uniform.
// Group 0 writes the float64 master A, the double-float copy (Ahi = the float
// compute copy, Alo), dA = A_new - ref (ref = A_p, or A_old when Arefhi is
// null) as float64 and float, and per-row ||dA||^2, ||A_new||^2
// (double-float).  With an update step size lam != 1 (Sec. 5.1) the new row
// is (1 - lam) A_old + lam a.
constexpr int kRB = 4;

__device__ __forceinline__ dfl dot2_val(dfl acc) { return fast_two_sum(acc.hi, acc.lo); }

__global__ void __launch_bounds__(256)
solve_inv_df_kernel(const float* __restrict__ rhs, double* __restrict__ A, float* __restrict__ Ahi,
                    float* __restrict__ Alo, const float* __restrict__ Arefhi,
                    const float* __restrict__ Areflo, double* __restrict__ dA,
                    float* __restrict__ dAc, const float2* __restrict__ Wg,
                    const float* __restrict__ Zg, float2* __restrict__ rownorm, int s, int R, int n,
                    double lam, const int* __restrict__ status) {
  extern __shared__ __align__(16) float2 smem[];
  const int RS = R | 1;
  float2* Ws = smem;
  const uint32_t wbytes = (uint32_t)(((size_t)R * RS * sizeof(float2) + 15) / 16 * 16);
  const uint32_t zbytes = Zg ? (uint32_t)(((size_t)R * R * sizeof(float) + 15) / 16 * 16) : 0u;
  float* Zs = reinterpret_cast<float*>(reinterpret_cast<char*>(smem) + wbytes);
  __shared__ __align__(8) uint64_t bar;
  __shared__ float2 bs[kRB][kMaxRank], ys[kRB][kMaxRank], hp[kRB][kMaxRank];
  __shared__ float as[kRB][kMaxRank];
  __shared__ float2 red[kRB][2][kMaxRank / 32];
  const bool failed = (status[0] >> n) & 1;
  const bool dense = (status[0] >> (16 + n)) & 1;   // W = diag(w^+)^(1/2) V^T, not L^-1
  const int Rp = (R + 31) / 32 * 32;
  const int h = threadIdx.x >= Rp;              // half of the terms
  const int r = threadIdx.x - h * Rp, lane = r & 31, warp = r >> 5, nwarp = Rp >> 5;
  const bool act = r < R;
  const int rr = act ? r : R - 1;               // padding threads read a valid row, store nothing
  const int m = (R + 1) / 2;                    // split point of the terms
  bool loaded = true;
  if (!failed) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                   "r"(wbytes + zbytes) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   ::"r"((uint32_t)__cvta_generic_to_shared(Ws)), "l"(Wg), "r"(wbytes), "r"(b) : "memory");
      if (Zg)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"((uint32_t)__cvta_generic_to_shared(Zs)), "l"(Zg), "r"(zbytes), "r"(b) : "memory");
    }
    __syncthreads();
    // bounded wait for the copies (phase 0)
    const unsigned long long t0 = clock64();
    while (true) {
      uint32_t done;
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                   " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(b) : "memory");
      if (done) break;
      if (clock64() - t0 > 4000000000ull) {
        loaded = false;
        break;
      }
    }
  }
  // every thread waited on the same barrier; a timeout anywhere reads as failure
  if (__syncthreads_or(!loaded)) {
    if (threadIdx.x == 0) atomicOr(const_cast<int*>(status) + 2, 1);
    return;
  }
  // y_r = sum_{c <= r} W_rc b_c: half 0 takes c < m, half 1 c >= m
  const int wend = dense ? R : min(R, 32 * warp + 32);   // L^-1 row r is zero beyond column r
  const int c1a = h ? m : 0, c1b = h ? wend : min(m, wend);
  // a_r = sum_{c >= r} W_cr y_c: half 0 takes c < m, half 1 c >= m
  const int wbeg = dense ? 0 : 32 * warp;
  const int c2a = h ? max(m, wbeg) : wbeg, c2b = h ? R : m;
  for (int y0 = blockIdx.x * kRB; y0 < s; y0 += gridDim.x * kRB) {
    float oh[kRB], ol[kRB];
    dfl a[kRB];
#pragma unroll
    for (int w = 0; w < kRB; w++) {
      const int y = min(y0 + w, s - 1);         // rows past the end repeat the last one (not stored)
      const int64_t o = (int64_t)y * R + rr;
      oh[w] = Ahi[o];
      ol[w] = Alo[o];
      a[w] = {rhs[o], 0.f};
      if (!h) as[w][rr] = oh[w];
    }
    if (failed) {
#pragma unroll
      for (int w = 0; w < kRB; w++) a[w] = {oh[w], ol[w]};
    } else {
      if (Zg) {
        __syncthreads();
        // second-order PP terms: b += A_old Z (float)
        float vz[kRB];
#pragma unroll
        for (int w = 0; w < kRB; w++) vz[w] = 0.f;
        for (int k = 0; k < R; k++) {
          const float zz = Zs[k * R + rr];
#pragma unroll
          for (int w = 0; w < kRB; w++) vz[w] = fmaf(as[w][k], zz, vz[w]);
        }
#pragma unroll
        for (int w = 0; w < kRB; w++) a[w] = df_add(a[w], dfl{vz[w], 0.f});
      }
      if (!h)
#pragma unroll
        for (int w = 0; w < kRB; w++) bs[w][rr] = pk(a[w]);
      __syncthreads();
      dfl acc[kRB];
#pragma unroll
      for (int w = 0; w < kRB; w++) acc[w] = {0.f, 0.f};
      const float2* wr = Ws + rr * RS;
#pragma unroll 2
      for (int c = c1a; c < c1b; c++) {
        const dfl wv = upk(wr[c]);
#pragma unroll
        for (int w = 0; w < kRB; w++) dot2_acc(acc[w], wv, upk(bs[w][c]));
      }
      if (h)
#pragma unroll
        for (int w = 0; w < kRB; w++) hp[w][rr] = pk(dot2_val(acc[w]));
      __syncthreads();
      if (!h)
#pragma unroll
        for (int w = 0; w < kRB; w++) ys[w][rr] = pk(df_add(dot2_val(acc[w]), upk(hp[w][rr])));
      __syncthreads();
#pragma unroll
      for (int w = 0; w < kRB; w++) acc[w] = {0.f, 0.f};
#pragma unroll 2
      for (int c = c2a; c < c2b; c++) {
        const dfl wv = upk(Ws[c * RS + rr]);
#pragma unroll
        for (int w = 0; w < kRB; w++) dot2_acc(acc[w], wv, upk(ys[w][c]));
      }
      if (h)
#pragma unroll
        for (int w = 0; w < kRB; w++) hp[w][rr] = pk(dot2_val(acc[w]));
      __syncthreads();
#pragma unroll
      for (int w = 0; w < kRB; w++) a[w] = df_add(dot2_val(acc[w]), upk(hp[w][rr]));
      if (lam != 1.0) {
        // update step size (Sec. 5.1): (1 - lam) A_old + lam a
        const dfl l1 = df_of(lam), l0 = df_of(1.0 - lam);
#pragma unroll
        for (int w = 0; w < kRB; w++) a[w] = df_add(df_mul(l1, a[w]), df_mul(l0, dfl{oh[w], ol[w]}));
      }
    }
    // outputs and per-row norms (group 0)
    if (!h) {
#pragma unroll
      for (int w = 0; w < kRB; w++) {
        const int y = y0 + w;
        dfl nd = {0.f, 0.f}, na = {0.f, 0.f};
        if (act && y < s) {
          const int64_t o = (int64_t)y * R + r;
          const dfl ref = Arefhi ? dfl{Arefhi[o], Areflo[o]} : dfl{oh[w], ol[w]};
          const dfl d = df_sub(a[w], ref);
          A[o] = df_dbl(a[w]);
          Ahi[o] = a[w].hi;
          Alo[o] = a[w].lo;
          dA[o] = df_dbl(d);
          dAc[o] = d.hi;
          nd = df_mul(d, d);
          na = df_mul(a[w], a[w]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          nd = df_add(nd, dfl{__shfl_xor_sync(0xffffffffu, nd.hi, off), __shfl_xor_sync(0xffffffffu, nd.lo, off)});
          na = df_add(na, dfl{__shfl_xor_sync(0xffffffffu, na.hi, off), __shfl_xor_sync(0xffffffffu, na.lo, off)});
        }
        if (lane == 0) {
          red[w][0][warp] = pk(nd);
          red[w][1][warp] = pk(na);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < kRB && y0 + (int)threadIdx.x < s) {
      const int w = threadIdx.x;
      dfl nd = upk(red[w][0][0]), na = upk(red[w][1][0]);
      for (int q = 1; q < nwarp; q++) {
        nd = df_add(nd, upk(red[w][0][q]));
        na = df_add(na, upk(red[w][1][q]));
      }
      rownorm[2 * (y0 + w)] = pk(nd);
      rownorm[2 * (y0 + w) + 1] = pk(na);
    }
    __syncthreads();                            // bs/ys/hp/as/red are reused by the next rows
  }
}

}  // namespace

// ---------------------------------------------------------------- host wrappers
cudaError_t setup_df_kernels() {
  const int RSmax = kMaxRank | 1;
  const int sv = (int)(kMaxRank * RSmax * sizeof(float2) + 16 + kMaxRank * kMaxRank * sizeof(float));
  cudaError_t e = cudaFuncSetAttribute(chol_inv_df_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)chol_inv_smem(kMaxRank));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(solve_inv_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pinv_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kMaxRank * RSmax * sizeof(double)));
  return e;
}

void split_df(const double* A, float* hi, float* lo, int64_t n, Launch L) {
  const int blocks = (int)std::min<int64_t>(cdiv(n, 256), 152 * 8);
  split_kernel<<<blocks, 256, 0, L.stream>>>(A, hi, lo, n);
  (*L.counter)++;
}

void gram_df(const float* Ahi, const float* Alo, const float* Aw, const float* dAw, double* S,
             float* Shi, float* Slo, float* W, bool withW, int s, int R, const float2* rownorm,
             double* scal, const float* ShiAll, const float* SloAll, int N, int n, int nn,
             float2* Gpk, Launch L) {
  const int nb = (R + 31) / 32;
  const int ntS = nb * (nb + 1) / 2;
  const int ntiles = withW ? ntS + nb * nb : ntS;
  // up to 8 CTAs per tile (a portable cluster), at least 16 rows each
  const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(8, cdiv(s, 16)));
  const int chunk = (int)cdiv(s, splits);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ntiles * splits);
  cfg.blockDim = dim3(256);
  cfg.stream = L.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = splits;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, gram_df_kernel, Ahi, Alo, Aw, dAw, s, R, nb, ntS, splits, chunk, S, Shi,
                     Slo, W, rownorm, scal, ShiAll, SloAll, N, n, nn, nn >= 0 ? Gpk : nullptr);
  (*L.counter)++;
}

void chol_df(const float* Shi, const float* Slo, const float* W, const float2* Gpk, int N, int n,
             int R, float2* Winv, float* Z, bool useV, int* status, Launch L) {
  const int T = R * (R + 1) / 2;
  // the chain CTA needs six warps (row threads in warps 1-3 and 5, the pivot
  // warp 4); the other CTAs use about one thread per eight packed entries
  const int threads = std::min(CPALS_CHOL_THREADS, std::max(192, (T / 8 + 31) / 32 * 32));
  chol_inv_df_kernel<<<5, threads, chol_inv_smem(R), L.stream>>>(Shi, Slo, W, Gpk, N, n, R, Winv,
                                                                 Z, useV ? 1 : 0, status);
  (*L.counter)++;
  pinv_df_kernel<<<1, 512, (size_t)R * (R | 1) * sizeof(double), L.stream>>>(Shi, Slo, Gpk, N, n, R,
                                                                             Winv, status);
  (*L.counter)++;
}

void solve_df(const float* rhs, double* A, float* Ahi, float* Alo, const float* Arefhi,
              const float* Areflo, double* dA, float* dAc, const float2* Winv, const float* Z,
              float2* rownorm, int s, int R, int n, double lam, const int* status, Launch L) {
  const size_t wb = ((size_t)R * (R | 1) * sizeof(float2) + 15) / 16 * 16;
  const size_t zb = Z ? ((size_t)R * R * sizeof(float) + 15) / 16 * 16 : 0;
  const int threads = 2 * ((R + 31) / 32 * 32);
  const int blocks = (int)std::min<int64_t>(cdiv(s, kRB), 152 * 2);
  solve_inv_df_kernel<<<blocks, threads, wb + zb, L.stream>>>(rhs, A, Ahi, Alo, Arefhi, Areflo, dA,
                                                              dAc, Winv, Z, rownorm, s, R, n,
                                                              lam, status);
  (*L.counter)++;
}

}  // namespace cpals
