// Double-float (hi + lo, two floats, 48-bit significand) kernels for the R x R
// normal-equation work of the FP32 and MIXED_BF16 modes (Sec. 2.3; Algorithm 1
// lines 5-10; Algorithm 3 lines 11-17).
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

#include "internal.h"

namespace cpals {

namespace {

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {   // requires |a| >= |b|
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  const dfl t = two_sum(x.lo, y.lo);
  const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const dfl c = two_prod(x.hi, y.hi);
  const float t0 = __fmul_rn(x.lo, y.lo);
  const float t1 = __fmaf_rn(x.hi, y.lo, t0);
  const float t2 = __fmaf_rn(x.lo, y.hi, t1);
  return fast_two_sum(c.hi, __fadd_rn(c.lo, t2));
}
// sqrt by one Newton step from the float square root (doubles the precision)
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  const float s = __fsqrt_rn(a.hi);
  const dfl d = df_sub(a, two_prod(s, s));
  return fast_two_sum(s, __fdiv_rn(d.hi, __fmul_rn(2.f, s)));
}
// reciprocal by one Newton step from the float reciprocal
__device__ __forceinline__ dfl df_recip(dfl a) {
  const float r = __frcp_rn(a.hi);
  const dfl d = df_sub(dfl{1.f, 0.f}, df_mul(a, dfl{r, 0.f}));
  return fast_two_sum(r, __fmul_rn(d.hi, r));
}
// "sloppy" double-word addition (one TwoSum): error bounded relative to
// |x| + |y| (a few units of 2^-48); used where that backward-error bound is
// what matters (the Cholesky trailing update)
__device__ __forceinline__ dfl df_add_fast(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
// 1/sqrt(a): float reciprocal square root refined by one Newton step in
// double-float, r = r0 + r0 (1 - a r0^2) / 2
__device__ __forceinline__ dfl df_rsqrt(dfl a) {
  const float r0 = rsqrtf(a.hi);
  const dfl r2 = two_prod(r0, r0);
  const dfl ar2 = df_mul(a, r2);
  const dfl e = df_sub(dfl{1.f, 0.f}, ar2);
  return fast_two_sum(r0, __fmul_rn(__fmul_rn(0.5f, r0), e.hi));
}
__device__ __forceinline__ dfl df_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_dbl(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ float2 pk(dfl a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ dfl upk(float2 a) { return {a.x, a.y}; }

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
// second-order PP terms use it).  One launch; the last CTA of each tile
// (ticket) reduces its split partials in split order with double-word adds.
__global__ void __launch_bounds__(256)
gram_df_kernel(const float* __restrict__ Ahi, const float* __restrict__ Alo,
               const float* __restrict__ Aw, const float* __restrict__ dAw, int s, int R, int nb,
               int ntS, int ntiles, int splits, int chunk, float2* __restrict__ part,
               int* __restrict__ tickets, double* __restrict__ S, float* __restrict__ Shi,
               float* __restrict__ Slo, float* __restrict__ W, const float2* __restrict__ rownorm,
               double* __restrict__ scal) {
  const int t = blockIdx.x % ntiles;
  const int z = blockIdx.x / ntiles;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int y0 = z * chunk, y1 = min(s, y0 + chunk);
  float2* p = part + ((int64_t)z * ntiles + t) * 1024;
  int ti, tj;
  __shared__ float Ah[32][33], Al[32][33], Bh[32][33], Bl[32][33];
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
    for (int q = 0; q < 4; q++) p[(ty + 8 * q) * 32 + tx] = pk(fast_two_sum(sh[q], sl[q]));
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
    for (int q = 0; q < 4; q++) p[(ty + 8 * q) * 32 + tx] = make_float2(acc[q], 0.f);
  }
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&tickets[t], 1) == splits - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int RR = R * R;
  for (int e = threadIdx.x; e < 1024; e += 256) {
    dfl acc = upk(__ldcg(part + (int64_t)t * 1024 + e));
    for (int zz = 1; zz < splits; zz++)
      acc = df_add(acc, upk(__ldcg(part + ((int64_t)zz * ntiles + t) * 1024 + e)));
    const int i = ti * 32 + e / 32, j = tj * 32 + e % 32;
    if (i < R && j < R) {
      if (t < ntS) {
        const double v = df_dbl(acc);
        S[i * R + j] = v;
        S[j * R + i] = v;
        Shi[i * R + j] = acc.hi;
        Shi[j * R + i] = acc.hi;
        Slo[i * R + j] = acc.lo;
        Slo[j * R + i] = acc.lo;
      } else {
        W[i * R + j] = acc.hi;
      }
    }
  }
  (void)RR;
  __shared__ int lastall;
  __syncthreads();
  if (threadIdx.x == 0) {
    tickets[t] = 0;
    lastall = (atomicAdd(&tickets[63], 1) == ntiles - 1);
  }
  __syncthreads();
  if (!lastall) return;
  // per-row ||dA||^2 and ||A||^2 (double-float) reduced in a fixed order
  __shared__ float2 rd[256], ra[256];
  dfl a = {0.f, 0.f}, b = {0.f, 0.f};
  for (int y = threadIdx.x; y < s; y += blockDim.x) {
    a = df_add(a, upk(__ldcg(rownorm + 2 * y)));
    b = df_add(b, upk(__ldcg(rownorm + 2 * y + 1)));
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
    tickets[63] = 0;
  }
}

// ---------------------------------------------------------------- Gamma + Cholesky
// One CTA: Gamma^(n) = Hadamard product of S^(k), k != n (double-float), then
// a right-looking Cholesky in shared memory (row stride RS = R|1) with one
// barrier per pivot.  The lower triangle is enumerated column-major,
// e(i, j) = j R - j(j-1)/2 + (i - j); thread t owns the entries e = t mod nt.
// At step k the entries still to update (columns > k) are the suffix
// e >= e(k+1, k+1) and column k-1 is the range [e(k-1,k-1), e(k,k)), so a
// thread only visits live entries.  Every thread takes 1/piv_k itself (no
// broadcast) and updates G_ij -= G_ik G_jk / piv_k from the unscaled column k;
// column k-1, which no thread reads at step k, is scaled to L then.
// Writes L (row stride RS, the layout the row solve copies in one bulk
// transfer) and the reciprocals of its diagonal.  With useV also the float
// matrix Z of the second-order terms (Eq. 3).
constexpr int kCholThreads = 1024;

__device__ __forceinline__ int col_start(int j, int R) { return j * R - j * (j - 1) / 2; }

__global__ void __launch_bounds__(kCholThreads, 1)
chol_df_kernel(const float* __restrict__ Shi, const float* __restrict__ Slo,
               const float* __restrict__ W, int N, int n, int R, float2* __restrict__ Lout,
               float2* __restrict__ invd, float* __restrict__ Z, int useV, int* __restrict__ status) {
  extern __shared__ float2 G[];
  __shared__ int colstart[kMaxRank + 2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int RR = R * R;
  const int RS = R | 1;
  for (int idx = tid; idx < RR; idx += nt) {
    const int i = idx / R, j = idx % R;
    if (j <= i) {
      dfl g = {1.f, 0.f};
      bool first = true;
      for (int k = 0; k < N; k++) {
        if (k == n) continue;
        const dfl sk = {Shi[(int64_t)k * RR + idx], Slo[(int64_t)k * RR + idx]};
        g = first ? sk : df_mul(g, sk);
        first = false;
      }
      G[i * RS + j] = pk(g);
    }
    if (useV) {
      float zz = 0.f;
      for (int a = 0; a < N; a++) {
        if (a == n) continue;
        for (int b = a + 1; b < N; b++) {
          if (b == n) continue;
          float h = W[(int64_t)a * RR + idx] * W[(int64_t)b * RR + idx];
          for (int k = 0; k < N; k++)
            if (k != a && k != b && k != n) h *= Shi[(int64_t)k * RR + idx];
          zz += h;
        }
      }
      Z[idx] = zz;
    }
  }
  for (int j = tid; j <= R + 1; j += nt) colstart[j] = col_start(min(j, R), R);
  __syncthreads();
  const int E = colstart[R];
  dfl ipiv_prev = {0.f, 0.f}, il_prev = {0.f, 0.f};
  for (int k = 0; k <= R; k++) {
    dfl il = {0.f, 0.f}, ipiv = {0.f, 0.f};
    if (k < R) {
      const dfl piv = upk(G[k * RS + k]);
      if (!(piv.hi > 0.f) || !isfinite(piv.hi)) {
        // every thread read the same pivot: the exit is uniform
        if (tid == 0) atomicOr(status, 1 << n);
        return;
      }
      il = df_rsqrt(piv);
      ipiv = df_mul(il, il);
      if (tid == 0) invd[k] = pk(il);
    }
    // scale column k-1 to L: its entries are a contiguous range
    if (k > 0) {
      const int e0 = colstart[k - 1], e1 = colstart[k];
      for (int e = e0 + tid; e < e1; e += nt) {
        const int i = (k - 1) + (e - e0);
        G[i * RS + (k - 1)] = pk(df_mul(upk(G[i * RS + (k - 1)]), il_prev));
      }
    }
    // trailing update of columns j > k
    if (k < R - 1) {
      const int es = colstart[k + 1];
      // first owned entry >= es; the column of entry e is the largest j with
      // colstart[j] <= e (root of j^2 - (2R+1) j + 2e, then exact fix-ups)
      const float b2 = (float)(2 * R + 1);
      for (int e = es + ((tid - es) % nt + nt) % nt; e < E; e += nt) {
        int j = (int)((b2 - sqrtf(fmaxf(b2 * b2 - 8.f * (float)e, 0.f))) * 0.5f);
        j = max(0, min(j, R - 1));
        while (j > 0 && colstart[j] > e) j--;
        while (colstart[j + 1] <= e) j++;
        const int i = j + (e - colstart[j]);
        const dfl gik = upk(G[i * RS + k]);
        const dfl gjk = upk(G[j * RS + k]);
        const dfl t = df_mul(df_mul(gik, gjk), ipiv);
        G[i * RS + j] = pk(df_add_fast(upk(G[i * RS + j]), df_neg(t)));
      }
    }
    il_prev = il;
    ipiv_prev = ipiv;
    __syncthreads();
  }
  (void)ipiv_prev;
  for (int idx = tid; idx < R * RS; idx += nt) {
    const int i = idx / RS, j = idx % RS;
    Lout[idx] = (j <= i && j < R) ? G[idx] : make_float2(0.f, 0.f);
  }
}

// ---------------------------------------------------------------- row solves
constexpr int kChunks = kMaxRank / 32;

template <typename V>
__device__ __forceinline__ V pick(const V (&v)[kChunks], int c) {
  V out = v[0];
#pragma unroll
  for (int i = 1; i < kChunks; i++)
    if (c == i) out = v[i];
  return out;
}
template <typename V>
__device__ __forceinline__ void put(V (&v)[kChunks], int c, V x) {
#pragma unroll
  for (int i = 0; i < kChunks; i++)
    if (c == i) v[i] = x;
}

// One warp per row y: b = rhs (+ A_old Z, float), forward substitution
// L z = b, back substitution L^T a = z, all in double-float.  Writes the
// float64 master A, the double-float copy (Ahi = the float compute copy, Alo),
// dA = A_new - ref (ref = A_p, or A_old when Arefhi is null) as float64 and
// float, and per-row ||dA||^2, ||A_new||^2 (double-float).
__global__ void __launch_bounds__(128)
solve_df_kernel(const float* __restrict__ rhs, double* __restrict__ A, float* __restrict__ Ahi,
                float* __restrict__ Alo, const float* __restrict__ Arefhi,
                const float* __restrict__ Areflo, double* __restrict__ dA, float* __restrict__ dAc,
                const float2* __restrict__ Lg, const float2* __restrict__ invg,
                const float* __restrict__ Zg, float2* __restrict__ rownorm, int s, int R, int n,
                const int* __restrict__ status) {
  extern __shared__ __align__(16) float2 smem[];
  const int RS = R | 1;
  float2* Ls = smem;
  const uint32_t lbytes = (uint32_t)(((size_t)R * RS * sizeof(float2) + 15) / 16 * 16);
  const uint32_t ibytes = (uint32_t)(((size_t)R * sizeof(float2) + 15) / 16 * 16);
  const uint32_t zbytes = Zg ? (uint32_t)(((size_t)R * R * sizeof(float) + 15) / 16 * 16) : 0u;
  float2* inv = reinterpret_cast<float2*>(reinterpret_cast<char*>(smem) + lbytes);
  float* Zs = reinterpret_cast<float*>(reinterpret_cast<char*>(smem) + lbytes + ibytes);
  __shared__ __align__(8) uint64_t bar;
  const bool failed = (status[0] >> n) & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  bool loaded = true;
  if (!failed) {
    // one bulk asynchronous copy per array (sizes are padded to 16 bytes in global memory)
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                   "r"(lbytes + ibytes + zbytes) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   ::"r"((uint32_t)__cvta_generic_to_shared(Ls)), "l"(Lg), "r"(lbytes), "r"(b) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   ::"r"((uint32_t)__cvta_generic_to_shared(inv)), "l"(invg), "r"(ibytes), "r"(b) : "memory");
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
  if (!loaded) {
    if (threadIdx.x == 0) atomicOr(const_cast<int*>(status) + 2, 1);
    return;
  }
  // two rows per warp, interleaved: the two substitutions are independent
  // instruction streams (latency hiding) and share every load of L
  constexpr int RPW = 2;
  for (int y0 = (blockIdx.x * nwarp + warp) * RPW; y0 < s; y0 += gridDim.x * nwarp * RPW) {
    float oh[RPW][kChunks], ol[RPW][kChunks];
    dfl b[RPW][kChunks];
#pragma unroll
    for (int w = 0; w < RPW; w++) {
      const int y = min(y0 + w, s - 1);      // a missing second row repeats the first (not stored)
#pragma unroll
      for (int c = 0; c < kChunks; c++) {
        const int r = lane + 32 * c;
        const bool v = r < R;
        oh[w][c] = v ? Ahi[(int64_t)y * R + r] : 0.f;
        ol[w][c] = v ? Alo[(int64_t)y * R + r] : 0.f;
        b[w][c] = {v ? rhs[(int64_t)y * R + r] : 0.f, 0.f};
      }
    }
    if (failed) {
#pragma unroll
      for (int w = 0; w < RPW; w++)
#pragma unroll
        for (int c = 0; c < kChunks; c++) b[w][c] = {oh[w][c], ol[w][c]};
    } else {
      if (Zg) {
        // second-order PP terms: b += A_old Z (float)
        float vz[RPW][kChunks];
#pragma unroll
        for (int w = 0; w < RPW; w++)
#pragma unroll
          for (int c = 0; c < kChunks; c++) vz[w][c] = 0.f;
        for (int k = 0; k < R; k++) {
          float ak[RPW];
#pragma unroll
          for (int w = 0; w < RPW; w++) ak[w] = __shfl_sync(0xffffffffu, pick(oh[w], k >> 5), k & 31);
#pragma unroll
          for (int c = 0; c < kChunks; c++) {
            const int r = lane + 32 * c;
            if (32 * c < R && r < R) {
              const float zz = Zs[k * R + r];
#pragma unroll
              for (int w = 0; w < RPW; w++) vz[w][c] = fmaf(ak[w], zz, vz[w][c]);
            }
          }
        }
#pragma unroll
        for (int w = 0; w < RPW; w++)
#pragma unroll
          for (int c = 0; c < kChunks; c++) b[w][c] = df_add(b[w][c], dfl{vz[w][c], 0.f});
      }
      // forward substitution L z = b (updates use the one-TwoSum addition:
      // backward error of a few 2^-48 relative to the operands)
      for (int i = 0; i < R; i++) {
        const int ci = i >> 5, li = i & 31;
        const dfl inv_i = upk(inv[i]);
        dfl zi[RPW];
#pragma unroll
        for (int w = 0; w < RPW; w++) {
          const dfl bi = pick(b[w], ci);
          const dfl src = {__shfl_sync(0xffffffffu, bi.hi, li), __shfl_sync(0xffffffffu, bi.lo, li)};
          zi[w] = df_mul(src, inv_i);
          if (lane == li) put(b[w], ci, zi[w]);
        }
#pragma unroll
        for (int c = 0; c < kChunks; c++) {
          if (32 * c + 31 <= i || 32 * c >= R) continue;
          const int r = lane + 32 * c;
          if (r > i && r < R) {
            const dfl l = upk(Ls[r * RS + i]);
#pragma unroll
            for (int w = 0; w < RPW; w++) b[w][c] = df_add_fast(b[w][c], df_neg(df_mul(l, zi[w])));
          }
        }
      }
      // back substitution L^T a = z
      for (int i = R - 1; i >= 0; i--) {
        const int ci = i >> 5, li = i & 31;
        const dfl inv_i = upk(inv[i]);
        dfl ai[RPW];
#pragma unroll
        for (int w = 0; w < RPW; w++) {
          const dfl bi = pick(b[w], ci);
          const dfl src = {__shfl_sync(0xffffffffu, bi.hi, li), __shfl_sync(0xffffffffu, bi.lo, li)};
          ai[w] = df_mul(src, inv_i);
          if (lane == li) put(b[w], ci, ai[w]);
        }
#pragma unroll
        for (int c = 0; c < kChunks; c++) {
          if (32 * c >= i) continue;
          const int r = lane + 32 * c;
          if (r < i) {
            const dfl l = upk(Ls[i * RS + r]);
#pragma unroll
            for (int w = 0; w < RPW; w++) b[w][c] = df_add_fast(b[w][c], df_neg(df_mul(l, ai[w])));
          }
        }
      }
    }
#pragma unroll
    for (int w = 0; w < RPW; w++) {
      const int y = y0 + w;
      if (y >= s) break;
      dfl nd = {0.f, 0.f}, na = {0.f, 0.f};
#pragma unroll
      for (int c = 0; c < kChunks; c++) {
        const int r = lane + 32 * c;
        if (r < R) {
          const int64_t o = (int64_t)y * R + r;
          const dfl ref = Arefhi ? dfl{Arefhi[o], Areflo[o]} : dfl{oh[w][c], ol[w][c]};
          const dfl d = df_sub(b[w][c], ref);
          A[o] = df_dbl(b[w][c]);
          Ahi[o] = b[w][c].hi;
          Alo[o] = b[w][c].lo;
          dA[o] = df_dbl(d);
          dAc[o] = d.hi;
          nd = df_add(nd, df_mul(d, d));
          na = df_add(na, df_mul(b[w][c], b[w][c]));
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        nd = df_add(nd, dfl{__shfl_xor_sync(0xffffffffu, nd.hi, off), __shfl_xor_sync(0xffffffffu, nd.lo, off)});
        na = df_add(na, dfl{__shfl_xor_sync(0xffffffffu, na.hi, off), __shfl_xor_sync(0xffffffffu, na.lo, off)});
      }
      if (lane == 0) {
        rownorm[2 * y] = pk(nd);
        rownorm[2 * y + 1] = pk(na);
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- host wrappers
cudaError_t setup_df_kernels() {
  const int RSmax = kMaxRank | 1;
  const int g = (int)(kMaxRank * RSmax * sizeof(float2));
  const int sv = (int)(kMaxRank * RSmax * sizeof(float2) + 16 + kMaxRank * sizeof(float2) +
                       kMaxRank * kMaxRank * sizeof(float));
  cudaError_t e =
      cudaFuncSetAttribute(chol_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, g);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(solve_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
  return e;
}

void split_df(const double* A, float* hi, float* lo, int64_t n, Launch L) {
  const int blocks = (int)std::min<int64_t>(cdiv(n, 256), 152 * 8);
  split_kernel<<<blocks, 256, 0, L.stream>>>(A, hi, lo, n);
  (*L.counter)++;
}

void gram_df(const float* Ahi, const float* Alo, const float* Aw, const float* dAw, double* S,
             float* Shi, float* Slo, float* W, bool withW, int s, int R, const float2* rownorm,
             double* scal, float2* partials, int* tickets, Launch L) {
  const int nb = (R + 31) / 32;
  const int ntS = nb * (nb + 1) / 2;
  const int ntiles = withW ? ntS + nb * nb : ntS;
  const int chunk = 32;
  const int splits = (int)cdiv(s, chunk);
  gram_df_kernel<<<ntiles * splits, 256, 0, L.stream>>>(Ahi, Alo, Aw, dAw, s, R, nb, ntS, ntiles,
                                                        splits, chunk, partials, tickets, S, Shi,
                                                        Slo, W, rownorm, scal);
  (*L.counter)++;
}

void chol_df(const float* Shi, const float* Slo, const float* W, int N, int n, int R,
             float2* Lout, float2* invd, float* Z, bool useV, int* status, Launch L) {
  const size_t smem = (size_t)R * (R | 1) * sizeof(float2);
  chol_df_kernel<<<1, kCholThreads, smem, L.stream>>>(Shi, Slo, W, N, n, R, Lout, invd, Z,
                                                      useV ? 1 : 0, status);
  (*L.counter)++;
}

void solve_df(const float* rhs, double* A, float* Ahi, float* Alo, const float* Arefhi,
              const float* Areflo, double* dA, float* dAc, const float2* Lf, const float2* invd,
              const float* Z, float2* rownorm, int s, int R, int n, const int* status, Launch L) {
  const size_t lb = ((size_t)R * (R | 1) * sizeof(float2) + 15) / 16 * 16;
  const size_t ib = ((size_t)R * sizeof(float2) + 15) / 16 * 16;
  const size_t zb = Z ? ((size_t)R * R * sizeof(float) + 15) / 16 * 16 : 0;
  const int warps = 2, rows_per_block = 2 * warps;      // two rows per warp
  const int blocks = (int)std::min<int64_t>(cdiv(s, rows_per_block), 152 * 2);
  solve_df_kernel<<<blocks, 32 * warps, lb + ib + zb, L.stream>>>(
      rhs, A, Ahi, Alo, Arefhi, Areflo, dA, dAc, Lf, invd, Z, rownorm, s, R, n, status);
  (*L.counter)++;
}

}  // namespace cpals
