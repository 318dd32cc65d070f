// Float64 kernels of the normal-equation update (Sec. 2.3, the normal-equation
// steps of Algorithms 1 and 3) and the fitness (Sec. 5).  R <= 128.
#include <algorithm>

#include "internal.h"
#include "jacobi.cuh"

namespace cpals {

namespace {

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

constexpr int kChunks = kMaxRank / 32;

__device__ __forceinline__ double pick(const double (&v)[kChunks], int c) {
  double out = v[0];
#pragma unroll
  for (int i = 1; i < kChunks; i++)
    if (c == i) out = v[i];
  return out;
}
__device__ __forceinline__ void put(double (&v)[kChunks], int c, double x) {
#pragma unroll
  for (int i = 0; i < kChunks; i++)
    if (c == i) v[i] = x;
}

// 1/sqrt(x) for the Cholesky pivots: the float estimate refined by two
// Newton-Raphson steps y <- y + y (1 - x y^2) / 2 in float64 (the float
// estimate's ~2^-23 relative error squares at each step, below float64's
// rounding after two); outside float's exponent range the float64 quotient
// is taken instead.  A float64 division and square root take ~1,100 cycles
// on GB300, this ~450.
__device__ __forceinline__ double rsqrt_refined(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
#pragma unroll
  for (int it = 0; it < 2; it++) {
    const double e = fma(-(x * y), y, 1.0);
    y = fma(0.5 * y, e, y);
  }
  return y;
}

// ---------------------------------------------------------------- Gamma^dagger
// Algorithm 1 writes the pseudo-inverse Gamma^dagger; the Cholesky route
// below covers a positive definite Gamma, and this fallback the rest: the
// symmetric eigendecomposition Gamma = V diag(w) V^T (cyclic Jacobi,
// sym_eig_jacobi), then Gamma^dagger = V diag(w^+) V^T with eigenvalues at or
// below 1e-13 of the largest dropped.  G (shared memory, row stride RS) is
// rebuilt from the Grams (the factorisation overwrote it); V lives in Pout,
// which receives Gamma^dagger at the end.  Returns false if Gamma has a
// non-finite entry.
static_assert(kMaxRank <= kJacobiMaxRank, "Jacobi scratch");

__device__ bool gamma_pinv(const double* __restrict__ S, int N, int n, int R, double* G,
                           double* __restrict__ Pout) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int RR = R * R, RS = R | 1;
  __shared__ double w[kMaxRank];
  int fin = 1;
  for (int idx = tid; idx < RR; idx += nt) {
    double g = 1.0;
    for (int k = 0; k < N; k++)
      if (k != n) g *= S[(int64_t)k * RR + idx];
    const int i = idx / R, j = idx % R;
    G[i * RS + j] = g;
    Pout[idx] = i == j ? 1.0 : 0.0;
    fin &= isfinite(g) ? 1 : 0;
  }
  if (!__syncthreads_and(fin)) return false;
  sym_eig_jacobi(G, RS, Pout, R, R);
  pinv_weights(G, RS, R, false, w);
  for (int idx = tid; idx < RR; idx += nt) {
    const int i = idx / R, j = idx % R;
    double acc = 0.0;
    for (int k = 0; k < R; k++) acc = fma(Pout[i * R + k] * w[k], Pout[j * R + k], acc);
    G[i * RS + j] = acc;
  }
  __syncthreads();
  for (int idx = tid; idx < RR; idx += nt) Pout[idx] = G[(idx / R) * RS + idx % R];
  return true;
}

// ---------------------------------------------------------------- Gamma + Cholesky (+ Z)
// One CTA: Gamma^(n) = Hadamard product of S^(k), k != n, then a right-looking
// Cholesky Gamma = L L^T in shared memory (row stride RS = R|1, odd, so that
// column accesses are free of bank conflicts); a Gamma that is not positive
// definite gets Gamma^dagger instead (gamma_pinv).  With useV also
// Z = sum_{i<j; i,j != n} W_i * W_j * (*_{k not in {i,j,n}} S_k) (Eq. 3's
// V terms: sum V^(n,i,j) = A^(n) Z).
__global__ void __launch_bounds__(512)
gamma_chol_kernel(const double* __restrict__ S, const double* __restrict__ W, int N, int n, int R,
                  double* __restrict__ Lout, double* __restrict__ Z, int useV,
                  int* __restrict__ status) {
  extern __shared__ double G[];
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int RR = R * R;
  const int RS = R | 1;
  for (int idx = tid; idx < RR; idx += nt) {
    double g = 1.0;
    for (int k = 0; k < N; k++)
      if (k != n) g *= S[(int64_t)k * RR + idx];
    G[(idx / R) * RS + idx % R] = g;
    if (useV) {
      double z = 0.0;
      for (int i = 0; i < N; i++) {
        if (i == n) continue;
        for (int j = i + 1; j < N; j++) {
          if (j == n) continue;
          double h = W[(int64_t)i * RR + idx] * W[(int64_t)j * RR + idx];
          for (int k = 0; k < N; k++)
            if (k != i && k != j && k != n) h *= S[(int64_t)k * RR + idx];
          z += h;
        }
      }
      Z[idx] = z;
    }
  }
  // the pivots' reciprocal square roots
  __shared__ double dinv[kMaxRank];
  if (tid == 0) {
    bad = 0;
    const double piv = G[0];
    if (!(piv > 0.0) || !isfinite(piv)) {
      bad = 1;
    } else {
      const double il = rsqrt_refined(piv);
      dinv[0] = il;
      G[0] = piv * il;
    }
  }
  __syncthreads();
  for (int k = 0; k < R && !bad; k++) {
    const double il = dinv[k];
    for (int i = k + 1 + tid; i < R; i += nt) G[i * RS + k] *= il;
    __syncthreads();
    if (warp == 0) {
      // lookahead: column k + 1 first, then its pivot's reciprocal square
      // root while the other warps update the rest of the trailing triangle
      if (k + 1 < R) {
        const double lk = G[(k + 1) * RS + k];
        for (int i = k + 1 + lane; i < R; i += 32) G[i * RS + k + 1] = fma(-G[i * RS + k], lk, G[i * RS + k + 1]);
        __syncwarp();
        if (lane == 0) {
          const double piv = G[(k + 1) * RS + k + 1];
          if (!(piv > 0.0) || !isfinite(piv)) {
            bad = 1;
          } else {
            const double il1 = rsqrt_refined(piv);
            dinv[k + 1] = il1;
            G[(k + 1) * RS + k + 1] = piv * il1;
          }
        }
      }
    } else {
      // rows i >= k + 2, columns k + 2 <= j <= i: one warp per row, lanes over j
      for (int i = k + 2 + warp - 1; i < R; i += nw - 1) {
        const double lik = G[i * RS + k];
        for (int j = k + 2 + lane; j <= i; j += 32) G[i * RS + j] = fma(-lik, G[j * RS + k], G[i * RS + j]);
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (bad) {
    // not positive definite: Gamma^dagger in place of the factor (status bit
    // 16 + n tells the row solve); a non-finite Gamma is an error (bit n)
    const bool ok = gamma_pinv(S, N, n, R, G, Lout);
    if (tid == 0) atomicOr(status, ok ? 1 << (16 + n) : 1 << n);
    return;
  }
  if (tid == 0) atomicAnd(status, ~(1 << (16 + n)));
  for (int idx = tid; idx < RR; idx += nt) {
    const int i = idx / R, j = idx % R;
    Lout[idx] = (j <= i) ? G[i * RS + j] : 0.0;
  }
}

// rhs2[y][r] = rhs[y][r] + sum_k A[y][k] Z[k][r]  (second-order PP terms), in the
// compute precision T (a second-order correction; float64 in FP64 mode).
template <typename T, typename TZ>
__global__ void __launch_bounds__(256)
vterm_kernel(const T* __restrict__ rhs, const T* __restrict__ A, const TZ* __restrict__ Z,
             T* __restrict__ out, int s, int R) {
  extern __shared__ unsigned char zsm[];
  T* Zs = reinterpret_cast<T*>(zsm);
  for (int i = threadIdx.x; i < R * R; i += blockDim.x) Zs[i] = (T)Z[i];
  __syncthreads();
  const int64_t n = (int64_t)s * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / R;
    const int r = (int)(i % R);
    T acc = rhs[i];
    const T* a = A + y * R;
    for (int k = 0; k < R; k++) acc = fma(a[k], Zs[k * R + r], acc);
    out[i] = acc;
  }
}

// ---------------------------------------------------------------- row solves
// One warp per row y: forward substitution L z = b, back substitution
// L^T a = z, i.e. a = b Gamma^{-1} (two triangular solves per row); with an
// update step size lam != 1 (Sec. 5.1) the new row is (1 - lam) A_old + lam a.
template <typename TR, typename T>
__global__ void __launch_bounds__(128)
solve_rows_kernel(const TR* __restrict__ rhs, double* __restrict__ A,
                  const double* __restrict__ Aref, double* __restrict__ dA,
                  const double* __restrict__ Lg, T* __restrict__ Ac, T* __restrict__ dAc,
                  double* __restrict__ rownorm, int s, int R, int n, double lam,
                  const int* __restrict__ status) {
  extern __shared__ double Ls[];   // R x RS lower factor (RS = R|1), then R inverse diagonals
  const int RS = R | 1;
  double* inv = Ls + R * RS;
  const bool failed = (status[0] >> n) & 1;
  const bool pinv = (status[0] >> (16 + n)) & 1;   // Lg holds Gamma^dagger (dense), not L
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  if (!failed) {
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) Ls[(idx / R) * RS + idx % R] = Lg[idx];
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += blockDim.x) inv[i] = 1.0 / Ls[i * RS + i];
    __syncthreads();
  }
  for (int y = blockIdx.x * nw + warp; y < s; y += gridDim.x * nw) {
    double b[kChunks], old[kChunks];
#pragma unroll
    for (int c = 0; c < kChunks; c++) {
      const int r = lane + 32 * c;
      old[c] = r < R ? A[(int64_t)y * R + r] : 0.0;
      b[c] = r < R ? (double)rhs[(int64_t)y * R + r] : 0.0;
    }
    if (failed) {
#pragma unroll
      for (int c = 0; c < kChunks; c++) b[c] = old[c];
    } else if (pinv) {
      // a = b Gamma^dagger
      double a[kChunks];
#pragma unroll
      for (int c = 0; c < kChunks; c++) a[c] = 0.0;
      for (int k = 0; k < R; k++) {
        const double bk = __shfl_sync(0xffffffffu, pick(b, k >> 5), k & 31);
#pragma unroll
        for (int c = 0; c < kChunks; c++) {
          const int r = lane + 32 * c;
          if (32 * c < R && r < R) a[c] = fma(bk, Ls[k * RS + r], a[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < kChunks; c++) b[c] = a[c];
      if (lam != 1.0)
#pragma unroll
        for (int c = 0; c < kChunks; c++) b[c] = (1.0 - lam) * old[c] + lam * b[c];
    } else {
      for (int i = 0; i < R; i++) {
        const int ci = i >> 5, li = i & 31;
        const double zi = __shfl_sync(0xffffffffu, pick(b, ci), li) * inv[i];
        if (lane == li) put(b, ci, zi);
#pragma unroll
        for (int c = 0; c < kChunks; c++) {
          if (32 * c + 31 <= i || 32 * c >= R) continue;     // warp-uniform: no lane of chunk c is updated
          const int r = lane + 32 * c;
          if (r > i && r < R) b[c] = fma(-Ls[r * RS + i], zi, b[c]);
        }
      }
      for (int i = R - 1; i >= 0; i--) {
        const int ci = i >> 5, li = i & 31;
        const double ai = __shfl_sync(0xffffffffu, pick(b, ci), li) * inv[i];
        if (lane == li) put(b, ci, ai);
#pragma unroll
        for (int c = 0; c < kChunks; c++) {
          if (32 * c >= i) continue;                          // warp-uniform
          const int r = lane + 32 * c;
          if (r < i) b[c] = fma(-Ls[i * RS + r], ai, b[c]);
        }
      }
      if (lam != 1.0)   // update step size (Sec. 5.1): (1 - lam) A_old + lam a
#pragma unroll
        for (int c = 0; c < kChunks; c++) b[c] = (1.0 - lam) * old[c] + lam * b[c];
    }
    double nd = 0.0, na = 0.0;
#pragma unroll
    for (int c = 0; c < kChunks; c++) {
      const int r = lane + 32 * c;
      if (r < R) {
        const int64_t o = (int64_t)y * R + r;
        const double ref = Aref ? Aref[o] : old[c];
        const double d = failed ? dA[o] : b[c] - ref;
        A[o] = b[c];
        dA[o] = d;
        Ac[o] = (T)b[c];
        dAc[o] = (T)d;
        nd = fma(d, d, nd);
        na = fma(b[c], b[c], na);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      nd += __shfl_xor_sync(0xffffffffu, nd, off);
      na += __shfl_xor_sync(0xffffffffu, na, off);
    }
    if (lane == 0) {
      rownorm[2 * y] = nd;
      rownorm[2 * y + 1] = na;
    }
  }
}

// ---------------------------------------------------------------- Grams
// One launch: CTA (z, t) forms the partial tile t over rows [z*chunk,
// (z+1)*chunk) and the last CTA to finish a tile (per-tile ticket) sums that
// tile's partials in split order (deterministic) and writes it.  Tile t < ntS
// is an upper block (ti <= tj) of S = A^T A (float64); the others are blocks
// of W = Aw^T dAw in the compute precision TW (W only feeds the second-order
// PP terms).  The CTA that finishes last overall also reduces the per-row
// norms.  Tickets are reset by their last CTA, ready for the next launch.
template <typename TW>
__global__ void __launch_bounds__(256)
gram_kernel(const double* __restrict__ A, const TW* __restrict__ Aw, const TW* __restrict__ dAw,
            int s, int R, int nb, int ntS, int ntiles, int splits, int chunk,
            double* __restrict__ part, int* __restrict__ tickets, double* __restrict__ S,
            double* __restrict__ W, const double* __restrict__ rownorm, double* __restrict__ scal) {
  const int t = blockIdx.x % ntiles;
  const int z = blockIdx.x / ntiles;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int y0 = z * chunk, y1 = min(s, y0 + chunk);
  double* p = part + ((int64_t)z * ntiles + t) * 1024;
  int ti, tj;
  if (t < ntS) {
    int tt = t;
    ti = 0;
    while (tt >= nb - ti) { tt -= nb - ti; ti++; }
    tj = ti + tt;
    __shared__ double As[32][33], Bs[32][33];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int yb = y0; yb < y1; yb += 32) {
      for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
        const int yy = idx / 32, c = idx % 32;
        const int y = yb + yy;
        const int ci = ti * 32 + c, cj = tj * 32 + c;
        As[yy][c] = (y < y1 && ci < R) ? A[(int64_t)y * R + ci] : 0.0;
        Bs[yy][c] = (y < y1 && cj < R) ? A[(int64_t)y * R + cj] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int yy = 0; yy < 32; yy++) {
        const double bj = Bs[yy][tx];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[q] = fma(As[yy][ty + 8 * q], bj, acc[q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; q++) p[(ty + 8 * q) * 32 + tx] = acc[q];
  } else {
    ti = (t - ntS) / nb;
    tj = (t - ntS) % nb;
    __shared__ TW Aws[32][33], Bws[32][33];
    TW acc[4] = {TW(0), TW(0), TW(0), TW(0)};
    for (int yb = y0; yb < y1; yb += 32) {
      for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
        const int yy = idx / 32, c = idx % 32;
        const int y = yb + yy;
        const int ci = ti * 32 + c, cj = tj * 32 + c;
        Aws[yy][c] = (y < y1 && ci < R) ? Aw[(int64_t)y * R + ci] : TW(0);
        Bws[yy][c] = (y < y1 && cj < R) ? dAw[(int64_t)y * R + cj] : TW(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int yy = 0; yy < 32; yy++) {
        const TW bj = Bws[yy][tx];
#pragma unroll
        for (int q = 0; q < 4; q++) acc[q] = fma(Aws[yy][ty + 8 * q], bj, acc[q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; q++) p[(ty + 8 * q) * 32 + tx] = (double)acc[q];
  }
  // ---- last CTA of this tile reduces it
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&tickets[t], 1) == splits - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = threadIdx.x; e < 1024; e += 256) {
    double acc = 0.0;
    for (int zz = 0; zz < splits; zz++) acc += __ldcg(part + ((int64_t)zz * ntiles + t) * 1024 + e);
    const int i = ti * 32 + e / 32, j = tj * 32 + e % 32;
    if (i < R && j < R) {
      if (t < ntS) {
        S[i * R + j] = acc;
        S[j * R + i] = acc;
      } else {
        W[i * R + j] = acc;
      }
    }
  }
  __shared__ int lastall;
  __syncthreads();
  if (threadIdx.x == 0) {
    tickets[t] = 0;
    lastall = (atomicAdd(&tickets[63], 1) == ntiles - 1);
  }
  __syncthreads();
  if (!lastall) return;
  // ---- the last tile to finish reduces the per-row norms
  __shared__ double rd[256], ra[256];
  double a = 0.0, bsum = 0.0;
  for (int y = threadIdx.x; y < s; y += blockDim.x) {
    a += __ldcg(rownorm + 2 * y);
    bsum += __ldcg(rownorm + 2 * y + 1);
  }
  rd[threadIdx.x] = a;
  ra[threadIdx.x] = bsum;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      rd[threadIdx.x] += rd[threadIdx.x + st];
      ra[threadIdx.x] += ra[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scal[0] = rd[0];
    scal[1] = ra[0];
    tickets[63] = 0;
  }
}

// ---------------------------------------------------------------- fitness
template <typename T>
__global__ void fitness_kernel(const T* __restrict__ rhs, const double* __restrict__ A,
                               const double* __restrict__ S, int N, int R, int s,
                               double* __restrict__ part, const double* __restrict__ normX2p,
                               double* __restrict__ out, int* __restrict__ ticket) {
  // per block: <M^(N), A^(N)> and sum of the Hadamard product of the Grams
  const int64_t n1 = (int64_t)s * R;
  const int RR = R * R;
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1;
       i += (int64_t)gridDim.x * blockDim.x)
    a = fma((double)rhs[i], A[i], a);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < RR; i += gridDim.x * blockDim.x) {
    double h = 1.0;
    for (int k = 0; k < N; k++) h *= S[(int64_t)k * RR + i];
    b += h;
  }
  __shared__ double ra[256], rb[256];
  __shared__ int last;
  ra[threadIdx.x] = a;
  rb[threadIdx.x] = b;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      ra[threadIdx.x] += ra[threadIdx.x + st];
      rb[threadIdx.x] += rb[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ra[0];
    part[2 * blockIdx.x + 1] = rb[0];
    __threadfence();
    last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  // the last block sums the partials in block order (deterministic) and
  // resets the ticket for the next launch
  __threadfence();
  a = 0.0;
  b = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  ra[threadIdx.x] = a;
  rb[threadIdx.x] = b;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      ra[threadIdx.x] += ra[threadIdx.x + st];
      rb[threadIdx.x] += rb[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double inner = ra[0], model = rb[0];
    const double normX2 = *normX2p;
    const double res2 = normX2 - 2.0 * inner + model;
    out[0] = 1.0 - sqrt(fmax(res2, 0.0)) / sqrt(normX2);
    out[1] = inner;
    out[2] = model;
    *ticket = 0;
  }
}

}  // namespace

// ---------------------------------------------------------------- host wrappers
cudaError_t setup_small_kernels() {
  const int RSmax = kMaxRank | 1;
  const int g = (int)(kMaxRank * RSmax * sizeof(double));
  const int sv = (int)((kMaxRank * RSmax + kMaxRank) * sizeof(double));
  const int vz = (int)(kMaxRank * kMaxRank * sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(gamma_chol_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, g);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(solve_rows_kernel<double, double>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(solve_rows_kernel<float, float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sv);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(vterm_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, vz);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(vterm_kernel<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, vz);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(vterm_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, vz);
  return e;
}

void gamma_chol(const double* S, const double* W, int N, int n, int R, double* Lout, double* Z,
                bool useV, int* status, Launch L) {
  const size_t smem = (size_t)R * (R | 1) * sizeof(double);
  gamma_chol_kernel<<<1, 512, smem, L.stream>>>(S, W, N, n, R, Lout, Z, useV ? 1 : 0, status);
  (*L.counter)++;
}

template <typename T>
static void solve_launch(const T* rhs, double* A, const double* Aref, double* dA, const double* Lf,
                         T* Ac, T* dAc, double* rownorm, int s, int R, int n, double lam,
                         const int* status, Launch L) {
  const size_t smem = (size_t)(R * (R | 1) + R) * sizeof(double);
  const int rows_per_block = 2;      // spread the rows over all SMs
  const int blocks = (int)std::min<int64_t>(cdiv(s, rows_per_block), 152 * 4);
  solve_rows_kernel<T, T><<<blocks, 32 * rows_per_block, smem, L.stream>>>(
      rhs, A, Aref, dA, Lf, Ac, dAc, rownorm, s, R, n, lam, status);
  (*L.counter)++;
}

template <typename T>
void solve_rows(const T* rhs, double* A, const double* Aref, double* dA, const double* Lf, T* Ac,
                T* dAc, double* rownorm, int s, int R, int n, double lam, const int* status,
                Launch L) {
  solve_launch<T>(rhs, A, Aref, dA, Lf, Ac, dAc, rownorm, s, R, n, lam, status, L);
}

template <typename T>
void vterm(const T* rhs, const T* A, const double* Z, T* out, int s, int R, Launch L) {
  const int64_t tot = (int64_t)s * R;
  vterm_kernel<T, double><<<(int)std::min<int64_t>(cdiv(tot, 256), 152 * 2), 256,
                            (size_t)R * R * sizeof(T), L.stream>>>(rhs, A, Z, out, s, R);
  (*L.counter)++;
}

void vterm_fz(const float* rhs, const float* A, const float* Z, float* out, int s, int R, Launch L) {
  const int64_t tot = (int64_t)s * R;
  vterm_kernel<float, float><<<(int)std::min<int64_t>(cdiv(tot, 256), 152 * 2), 256,
                               (size_t)R * R * sizeof(float), L.stream>>>(rhs, A, Z, out, s, R);
  (*L.counter)++;
}

template <typename T>
void solve_rows_v(const T* rhs, double* A, const double* Aref, double* dA, const double* Lf,
                  const double* Z, T* rhs2, T* Ac, T* dAc, double* rownorm, int s, int R, int n,
                  double lam, const int* status, Launch L) {
  vterm<T>(rhs, Ac, Z, rhs2, s, R, L);
  solve_launch<T>(rhs2, A, Aref, dA, Lf, Ac, dAc, rownorm, s, R, n, lam, status, L);
}

template <typename T>
void gram_update(const double* A, const T* Ac, const T* dAc, double* S, double* W, bool withW,
                 int s, int R, const double* rownorm, double* scal, double* partials, int* tickets,
                 Launch L) {
  const int nb = (R + 31) / 32;
  const int ntS = nb * (nb + 1) / 2;
  const int ntiles = withW ? ntS + nb * nb : ntS;
  const int chunk = 32;
  const int splits = (int)cdiv(s, chunk);
  gram_kernel<T><<<ntiles * splits, 256, 0, L.stream>>>(A, Ac, dAc, s, R, nb, ntS, ntiles, splits,
                                                        chunk, partials, tickets, S, W, rownorm,
                                                        scal);
  (*L.counter) += 1;
}

template <typename T>
void fitness(const T* rhs, const double* A, const double* S, int N, int R, int s,
             const double* normX2, double* out, double* partials, int* ticket, Launch L) {
  fitness_kernel<T><<<128, 256, 0, L.stream>>>(rhs, A, S, N, R, s, partials, normX2, out, ticket);
  (*L.counter) += 1;
}

#define INST(T)                                                                                 \
  template void solve_rows<T>(const T*, double*, const double*, double*, const double*, T*, T*, \
                              double*, int, int, int, double, const int*, Launch);              \
  template void solve_rows_v<T>(const T*, double*, const double*, double*, const double*,       \
                                const double*, T*, T*, T*, double*, int, int, int, double,      \
                                const int*, Launch);                                            \
  template void vterm<T>(const T*, const T*, const double*, T*, int, int, Launch);              \
  template void gram_update<T>(const double*, const T*, const T*, double*, double*, bool, int,  \
                               int, const double*, double*, double*, int*, Launch);             \
  template void fitness<T>(const T*, const double*, const double*, int, int, int,               \
                           const double*, double*, double*, int*, Launch);
INST(double)
INST(float)
#undef INST

}  // namespace cpals
