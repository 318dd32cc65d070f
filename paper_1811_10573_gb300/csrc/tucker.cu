// Tucker-ALS (HOOI, Algorithm 2) and pairwise-perturbation Tucker-ALS
// (Algorithm 4) for tensors of order 3 to 8 in IEEE float64.  Order 3 has the
// tuned layouts below; higher orders use the generic contraction chains of
// the "order N > 3" section.
//
// Order-3 sweep (Sec. 2.4 with the dimension tree of Sec. 2.5):
//   T  = X x_3 A3        [x1][x2][r3]   first level for modes 1 and 2
//   Y1 = T x_2 A2        [x1][r3][r2]
//   Y2 = T x_1 A1        [x2][r3][r1]   (A1 already updated)
//   U  = X x_1 A1        [x2][x3][r1]   first level for mode 3
//   Y3 = U x_2 A2        [x3][r1][r2]
//   G  = Y3 x_3 A3       [r1][r2][r3]
// (x_n A: contraction of mode n with the rows of A; 1-based in this comment.)
// Each factor update takes the R_n leading eigenvectors of the Gram matrix
// W = Y_(n) Y_(n)^T (the paper's reading of the leading left singular
// vectors) by subspace iteration started from the current factor (the
// W-products orthonormalised by Cholesky QR), then a Rayleigh-Ritz step
// whose R_n x R_n eigenproblem is solved by parallel cyclic Jacobi on one
// CTA; eigenvectors in decreasing eigenvalue order, each column signed to
// a non-negative inner product with the column it replaces.
//
// PP (Sec. 3.1.2): operators Y_p^(i,n) = X x_k A_p^(k) (k the third mode)
// and Y_p^(n); a PP sweep forms Y~^(n) = Y_p^(n) + sum_i Y_p^(i,n) x_i dA^(i)
// in the layouts above and updates as in ALS.  Fitness: 1 - sqrt(||X||^2 -
// ||G||^2) / ||X|| (orthonormal factors).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cpals.h"
#include "internal.h"

namespace cpals {
namespace {

inline int64_t cdivt(int64_t a, int64_t b) { return (a + b - 1) / b; }
constexpr int kTuckerMaxRank = 48;

// W[i][j] = sum_k Y[i K + k] Y[j K + k], 16 x 16 output tiles (one output per
// thread), K in chunks of 16; upper tiles only, mirrored on store.
__global__ void __launch_bounds__(256) syrk_kernel(const double* __restrict__ Y, int s, int K,
                                                   double* __restrict__ W) {
  __shared__ double a[16][17], b[16][17];
  const int ti = blockIdx.y * 16, tj = blockIdx.x * 16;
  if (tj < ti) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int k = k0 + tx;
    a[ty][tx] = (ti + ty < s && k < K) ? Y[(int64_t)(ti + ty) * K + k] : 0.0;
    b[ty][tx] = (tj + ty < s && k < K) ? Y[(int64_t)(tj + ty) * K + k] : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; q++) acc = fma(a[ty][q], b[tx][q], acc);
    __syncthreads();
  }
  const int i = ti + ty, j = tj + tx;
  if (i < s && j < s) {
    W[(int64_t)i * s + j] = acc;
    W[(int64_t)j * s + i] = acc;
  }
}

// out[i][c] = sum_k P[i K + k] B[k R + c] for R <= 48 columns, one CTA per
// row: warp w takes the 32-wide k chunks w, w + 8, ..., lanes own columns c
// and c + 32 with two accumulation chains each (the FP64 pipe has a long
// latency, so the row is spread over 8 warps); the warps' sums are added in
// warp order.
__global__ void __launch_bounds__(256) rowmm_kernel(const double* __restrict__ P,
                                                    const double* __restrict__ B, int K, int R,
                                                    double* __restrict__ out,
                                                    const int* __restrict__ skip) {
  if (skip && *skip) return;                 // the subspace iteration has converged
  __shared__ double red[8][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = blockIdx.x;
  const bool c0 = lane < R, c1 = lane + 32 < R;
  double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
  for (int k0 = w * 32; k0 < K; k0 += 256) {
    const int n = min(32, K - k0);
    const double pv = lane < n ? P[i * K + k0 + lane] : 0.0;
    const double* Bk = B + (int64_t)k0 * R;
    if (n == 32) {
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const double p0 = __shfl_sync(0xffffffffu, pv, j), p1 = __shfl_sync(0xffffffffu, pv, j + 1);
        if (c0) {
          a0 = fma(p0, __ldg(Bk + j * R + lane), a0);
          b0 = fma(p1, __ldg(Bk + (j + 1) * R + lane), b0);
        }
        if (c1) {
          a1 = fma(p0, __ldg(Bk + j * R + lane + 32), a1);
          b1 = fma(p1, __ldg(Bk + (j + 1) * R + lane + 32), b1);
        }
      }
    } else {
      for (int j = 0; j < n; j++) {
        const double p0 = __shfl_sync(0xffffffffu, pv, j);
        if (c0) a0 = fma(p0, __ldg(Bk + j * R + lane), a0);
        if (c1) a1 = fma(p0, __ldg(Bk + j * R + lane + 32), a1);
      }
    }
  }
  red[w][lane] = a0 + b0;
  red[w][lane + 32] = a1 + b1;
  __syncthreads();
  if (w == 0) {
    double v0 = 0.0, v1 = 0.0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      v0 += red[q][lane];
      v1 += red[q][lane + 32];
    }
    if (c0) out[i * R + lane] = v0;
    if (c1) out[i * R + lane + 32] = v1;
  }
}

// Batched small contraction out[b][m][r] = sum_k in[(b K + k) M + m] B[k R + r]
// for M, R <= 48 (the second-level TTMs and PP terms whose kept mode is a
// rank): one CTA per b owns its M x R outputs exactly (no padded FMAs on the
// FP64 pipe); 16 k at a time staged in shared memory, each output summed in
// k order.
__global__ void __launch_bounds__(256) bsmall_kernel(const double* __restrict__ in,
                                                     const double* __restrict__ B, int K, int M,
                                                     int R, double* __restrict__ out) {
  constexpr int kQ = (kTuckerMaxRank * kTuckerMaxRank + 255) / 256;
  __shared__ double is[16][kTuckerMaxRank], bs[16][kTuckerMaxRank];
  const double* inb = in + (int64_t)blockIdx.x * K * M;
  const int MR = M * R;
  double acc[kQ];
#pragma unroll
  for (int q = 0; q < kQ; q++) acc[q] = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int n = min(16, K - k0);
    for (int e = threadIdx.x; e < 16 * M; e += blockDim.x) {
      const int kk = e / M, m = e % M;
      is[kk][m] = kk < n ? inb[(int64_t)(k0 + kk) * M + m] : 0.0;
    }
    for (int e = threadIdx.x; e < 16 * R; e += blockDim.x) {
      const int kk = e / R, r = e % R;
      bs[kk][r] = kk < n ? B[(int64_t)(k0 + kk) * R + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kQ; q++) {
      const int e = threadIdx.x + 256 * q;
      if (e < MR) {
        const int m = e / R, r = e % R;
        double v = acc[q];
        for (int kk = 0; kk < n; kk++) v = fma(is[kk][m], bs[kk][r], v);
        acc[q] = v;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kQ; q++) {
    const int e = threadIdx.x + 256 * q;
    if (e < MR) out[(int64_t)blockIdx.x * MR + e] = acc[q];
  }
}

// part[blk][a][c] = sum over the block's rows i of P[i R + a] Q[i R + c]
// (rows_per_block consecutive rows; 32 rows staged in shared memory at a time)
__global__ void __launch_bounds__(256) atb_part_kernel(const double* __restrict__ P,
                                                       const double* __restrict__ Q, int s, int R,
                                                       int rows_per_block, double* __restrict__ part,
                                                       const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double ps[32][kTuckerMaxRank + 1], qs[32][kTuckerMaxRank + 1];
  const int r0 = blockIdx.x * rows_per_block, r1 = min(s, r0 + rows_per_block);
  const int RR = R * R;
  double acc[(kTuckerMaxRank * kTuckerMaxRank + 255) / 256];
#pragma unroll
  for (int q = 0; q < (kTuckerMaxRank * kTuckerMaxRank + 255) / 256; q++) acc[q] = 0.0;
  for (int i0 = r0; i0 < r1; i0 += 32) {
    const int n = min(32, r1 - i0);
    for (int e = threadIdx.x; e < 32 * R; e += blockDim.x) {
      const int i = e / R, c = e % R;
      ps[i][c] = i < n ? P[(int64_t)(i0 + i) * R + c] : 0.0;
      qs[i][c] = i < n ? Q[(int64_t)(i0 + i) * R + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (kTuckerMaxRank * kTuckerMaxRank + 255) / 256; q++) {
      const int e = threadIdx.x + 256 * q;
      if (e < RR) {
        const int a = e / R, c = e % R;
        double v = acc[q];
        for (int i = 0; i < n; i++) v = fma(ps[i][a], qs[i][c], v);
        acc[q] = v;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < (kTuckerMaxRank * kTuckerMaxRank + 255) / 256; q++) {
    const int e = threadIdx.x + 256 * q;
    if (e < RR) part[(int64_t)blockIdx.x * RR + e] = acc[q];
  }
}

// Cholesky QR step Q = Z L^-T with Z^T Z = L L^T: every CTA sums the nb
// partial Grams in block order, factors the R x R matrix in shared memory
// (redundantly; CTA 0 reports a non-positive pivot in bit 0 of *status),
// then solves q L^T = z for its rows (one warp per row).  Z and Q may alias.
__global__ void __launch_bounds__(256) cholqr_kernel(const double* __restrict__ part, int nb,
                                                     const double* Z, int s, int R, double* Q,
                                                     int* __restrict__ status,
                                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double L[kTuckerMaxRank][kTuckerMaxRank + 1];
  __shared__ double dinv[kTuckerMaxRank];
  const int RR = R * R;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < nb; b++) v += part[(int64_t)b * RR + e];
    L[e / R][e % R] = v;
  }
  __syncthreads();
  for (int k = 0; k < R; k++) {
    if (threadIdx.x == 0) {
      const double d = L[k][k];
      if (!(d > 0.0) && blockIdx.x == 0) atomicOr(status, 1);
      const double ri = rsqrt(fmax(d, 1e-300));
      L[k][k] = fmax(d, 1e-300) * ri;        // sqrt(d) = d / sqrt(d)
      dinv[k] = ri;
    }
    __syncthreads();
    const double di = dinv[k];
    for (int i = k + 1 + threadIdx.x; i < R; i += blockDim.x) L[i][k] *= di;
    __syncthreads();
    const int w = R - k - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int i = k + 1 + e / w, j = k + 1 + e % w;
      if (j <= i) L[i][j] = fma(-L[i][k], L[j][k], L[i][j]);
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = blockIdx.x * nw + warp; i < s; i += gridDim.x * nw) {
    double z0 = lane < R ? Z[(int64_t)i * R + lane] : 0.0;
    double z1 = lane + 32 < R ? Z[(int64_t)i * R + lane + 32] : 0.0;
    for (int k = 0; k < R; k++) {
      const double zk = __shfl_sync(0xffffffffu, k < 32 ? z0 : z1, k & 31) * dinv[k];
      if (k < 32) { if (lane == k) z0 = zk; } else { if (lane == k - 32) z1 = zk; }
      if (lane > k && lane < R) z0 = fma(-L[lane][k], zk, z0);
      if (lane + 32 > k && lane + 32 < R) z1 = fma(-L[lane + 32][k], zk, z1);
    }
    if (lane < R) Q[(int64_t)i * R + lane] = z0;
    if (lane + 32 < R) Q[(int64_t)i * R + lane + 32] = z1;
  }
}

// Convergence test of the subspace iteration: with Z = W Q and H = Q^T Z
// (the sum of nb partials), the invariance residual ||Z - Q H||_F^2 against
// ||Z||_F^2.  Every CTA sums the partials in block order and takes rows (one
// warp per row); the last CTA to finish adds the CTAs' sums in block order and
// sets *done when residual^2 <= tol2 * ||Z||^2, then re-arms the ticket.
__global__ void __launch_bounds__(256) resid_kernel(const double* __restrict__ part, int nb,
                                                    const double* __restrict__ Q,
                                                    const double* __restrict__ Z, int s, int R,
                                                    double tol2, double* __restrict__ rpart,
                                                    int* __restrict__ ticket, int* __restrict__ done) {
  if (*done) return;
  __shared__ double H[kTuckerMaxRank][kTuckerMaxRank + 1];
  __shared__ double red[2][8];
  __shared__ bool last;
  const int RR = R * R;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < nb; b++) v += part[(int64_t)b * RR + e];
    H[e / R][e % R] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double r2 = 0.0, z2 = 0.0;
  for (int i = blockIdx.x * nw + warp; i < s; i += gridDim.x * nw) {
    const double q0 = lane < R ? Q[(int64_t)i * R + lane] : 0.0;
    const double q1 = lane + 32 < R ? Q[(int64_t)i * R + lane + 32] : 0.0;
    const double z0 = lane < R ? Z[(int64_t)i * R + lane] : 0.0;
    const double z1 = lane + 32 < R ? Z[(int64_t)i * R + lane + 32] : 0.0;
    double a0 = 0.0, a1 = 0.0;
    for (int k = 0; k < R; k++) {
      const double qk = __shfl_sync(0xffffffffu, k < 32 ? q0 : q1, k & 31);
      if (lane < R) a0 = fma(qk, H[k][lane], a0);
      if (lane + 32 < R) a1 = fma(qk, H[k][lane + 32], a1);
    }
    const double d0 = z0 - a0, d1 = z1 - a1;
    r2 = fma(d0, d0, fma(d1, d1, r2));
    z2 = fma(z0, z0, fma(z1, z1, z2));
  }
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    z2 += __shfl_xor_sync(0xffffffffu, z2, o);
  }
  if (lane == 0) {
    red[0][warp] = r2;
    red[1][warp] = z2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nw; w++) {
      a += red[0][w];
      b += red[1][w];
    }
    rpart[2 * blockIdx.x] = a;
    rpart[2 * blockIdx.x + 1] = b;
    __threadfence();
    last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const volatile double* vp = rpart;
    double a = 0.0, b = 0.0;
    for (int blk = 0; blk < (int)gridDim.x; blk++) {
      a += vp[2 * blk];
      b += vp[2 * blk + 1];
    }
    if (a <= tol2 * b) *done = 1;
    *ticket = 0;
  }
}

// Eigen-decomposition of the symmetric R x R matrix H = sum of nb partials
// (one CTA): parallel cyclic Jacobi (round-robin pairing, R/2 disjoint
// rotations per step) until the off-diagonal sum of squares is below 1e-30
// of the diagonal one (at most 16 sweeps), then V's columns sorted by
// decreasing eigenvalue.
__global__ void __launch_bounds__(256) jacobi_kernel(const double* __restrict__ part, int nb, int R,
                                                     double* __restrict__ Vout,
                                                     double* __restrict__ lam_out) {
  __shared__ double A[kTuckerMaxRank][kTuckerMaxRank + 1], V[kTuckerMaxRank][kTuckerMaxRank + 1];
  __shared__ double cs[kTuckerMaxRank / 2][2];
  __shared__ int pp[kTuckerMaxRank / 2][2];
  __shared__ int perm[kTuckerMaxRank + 1];
  __shared__ double lam[kTuckerMaxRank];
  const int Re = R + (R & 1);                // even number of slots (a dummy when R is odd)
  __shared__ double red[2][8];
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double h = 0.0;
    for (int b = 0; b < nb; b++) h += part[(int64_t)b * R * R + e];
    A[e / R][e % R] = h;
    V[e / R][e % R] = (e / R == e % R) ? 1.0 : 0.0;
  }
  for (int i = threadIdx.x; i < Re; i += blockDim.x) perm[i] = i;
  __syncthreads();
  for (int sweep = 0; sweep < 16; sweep++) {
    double off = 0.0, dg = 0.0;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
      const double v = A[e / R][e % R];
      if (e / R == e % R) dg = fma(v, v, dg);
      else off = fma(v, v, off);
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dg += __shfl_xor_sync(0xffffffffu, dg, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = off;
      red[1][threadIdx.x >> 5] = dg;
    }
    __syncthreads();
    double to = 0.0, td = 0.0;
    for (int w = 0; w < 8; w++) {
      to += red[0][w];
      td += red[1][w];
    }
    __syncthreads();
    if (to <= 1e-30 * td) break;
    for (int step = 0; step < Re - 1; step++) {
      // pairs of this step: (perm[k], perm[Re-1-k])
      for (int k = threadIdx.x; k < Re / 2; k += blockDim.x) {
        int p = perm[k], q = perm[Re - 1 - k];
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, sn = 0.0;
        if (q < R) {
          const double apq = A[p][q];
          if (apq != 0.0) {
            // tan of the rotation angle: the smaller root of t^2 + 2 tau t - 1 = 0
            const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
            double t;
            if (fabs(tau) > 1e100) {
              t = 0.5 / tau;
            } else {
              const double u = fma(tau, tau, 1.0);
              t = copysign(1.0, tau) / fma(u, rsqrt(u), fabs(tau));   // sqrt(u) = u / sqrt(u)
            }
            c = rsqrt(fma(t, t, 1.0));
            sn = t * c;
          }
        }
        pp[k][0] = p;
        pp[k][1] = q;
        cs[k][0] = c;
        cs[k][1] = sn;
      }
      __syncthreads();
      // rows: A <- J^T A (each pair's two rows, all columns)
      for (int e = threadIdx.x; e < (Re / 2) * R; e += blockDim.x) {
        const int k = e / R, j = e % R, p = pp[k][0], q = pp[k][1];
        if (q >= R) continue;
        const double c = cs[k][0], sn = cs[k][1];
        const double ap = A[p][j], aq = A[q][j];
        A[p][j] = c * ap - sn * aq;
        A[q][j] = sn * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = threadIdx.x; e < (Re / 2) * R; e += blockDim.x) {
        const int k = e / R, i = e % R, p = pp[k][0], q = pp[k][1];
        if (q >= R) continue;
        const double c = cs[k][0], sn = cs[k][1];
        const double ap = A[i][p], aq = A[i][q];
        A[i][p] = c * ap - sn * aq;
        A[i][q] = sn * ap + c * aq;
        const double vp = V[i][p], vq = V[i][q];
        V[i][p] = c * vp - sn * vq;
        V[i][q] = sn * vp + c * vq;
      }
      __syncthreads();
      // next round-robin arrangement: slot 0 fixed, the others rotate
      if (threadIdx.x == 0) {
        const int last = perm[Re - 1];
        for (int i = Re - 1; i > 1; i--) perm[i] = perm[i - 1];
        perm[1] = last;
      }
      __syncthreads();
    }
  }
  // sort by decreasing eigenvalue (selection by rank; ties keep index order)
  for (int i = threadIdx.x; i < R; i += blockDim.x) lam[i] = A[i][i];
  __syncthreads();
  for (int i = threadIdx.x; i < R; i += blockDim.x) {
    int rank = 0;
    for (int j = 0; j < R; j++)
      if (lam[j] > lam[i] || (lam[j] == lam[i] && j < i)) rank++;
    lam_out[rank] = lam[i];
    for (int r = 0; r < R; r++) Vout[r * R + rank] = V[r][i];
  }
}

// A_new[:, r] = Q V[:, r], signed to a non-negative inner product with
// A_old[:, r]; one CTA per column.  dA = A_new - A_ref (ref = A_old, or A_p
// in PP sweeps); per-column ||dA||^2 and ||A_new||^2 into part[2 r], [2 r + 1].
__global__ void __launch_bounds__(256) qv_sign_kernel(const double* __restrict__ Q,
                                                      const double* __restrict__ V, int s, int R,
                                                      double* __restrict__ A,
                                                      const double* __restrict__ Aref,
                                                      double* __restrict__ dA,
                                                      double* __restrict__ part) {
  const int r = blockIdx.x;
  __shared__ double red[256];
  __shared__ double sgn;
  double dot = 0.0;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double a = 0.0;
    for (int k = 0; k < R; k++) a = fma(Q[(int64_t)i * R + k], V[k * R + r], a);
    dot = fma(a, A[(int64_t)i * R + r], dot);
  }
  red[threadIdx.x] = dot;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) sgn = red[0] < 0.0 ? -1.0 : 1.0;
  __syncthreads();
  double nd = 0.0, na = 0.0;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double a = 0.0;
    for (int k = 0; k < R; k++) a = fma(Q[(int64_t)i * R + k], V[k * R + r], a);
    a *= sgn;
    const double d = a - (Aref ? Aref[(int64_t)i * R + r] : A[(int64_t)i * R + r]);
    dA[(int64_t)i * R + r] = d;
    A[(int64_t)i * R + r] = a;
    nd = fma(d, d, nd);
    na = fma(a, a, na);
  }
  __syncthreads();
  red[threadIdx.x] = nd;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[2 * r] = red[0];
  __syncthreads();
  red[threadIdx.x] = na;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[2 * r + 1] = red[0];
}

// out[i] = in[i] (copy) or out[i] += in[i]
__global__ void axpy_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t n,
                            int add) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = add ? out[i] + in[i] : in[i];
}

// out[b][i][j] += in[b][j][i]  (i < P, j < Qd)
__global__ void add_transposed_kernel(const double* __restrict__ in, double* __restrict__ out,
                                      int64_t B, int P, int Qd) {
  const int64_t n = B * P * Qd;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / ((int64_t)P * Qd);
    const int rem = (int)(e % ((int64_t)P * Qd));
    const int i = rem / Qd, j = rem % Qd;
    out[e] += in[b * P * Qd + (int64_t)j * P + i];
  }
}

// Xb[i] = bf16(X[i]) (through float, round to nearest)
// out[x][a][r][b] (=, or += with add) in[x][a][b][r]: moves the rank index r
// of a contracted mode from the end of the layout to its place among the
// other rank indices (order N > 3: the PP terms and M_p^(n))
__global__ void permute_rank_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t nx,
                                    int64_t na, int nr, int64_t nb, int add) {
  const int64_t total = nx * na * nr * nb;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = o % nb;
    const int64_t r = (o / nb) % nr;
    const int64_t xa = o / (nb * nr);          // x * na + a
    const double v = in[(xa * nb + b) * nr + r];
    out[o] = add ? out[o] + v : v;
  }
}

__global__ void to_bf16_kernel(const double* __restrict__ X, __nv_bfloat16* __restrict__ Xb, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    Xb[i] = __float2bfloat16_rn((float)X[i]);
}

// Tensor-core B operand of a factor A (K x R, row-major): two planes of Rpad
// rows x Kstride, Bt[r][k] = hi(A[k][r]) and Bt[Rpad Kstride + r Kstride + k]
// = lo = bf16(a - hi) with a = float(A[k][r]); zero padding.
__global__ void factor_bt_kernel(const double* __restrict__ A, int64_t K, int R, int Rpad,
                                 int64_t Kstride, __nv_bfloat16* __restrict__ Bt) {
  const int64_t n = (int64_t)Rpad * Kstride;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / Kstride);
    const int64_t k = e % Kstride;
    const float a = (r < R && k < K) ? (float)A[k * R + r] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(a);
    Bt[e] = hi;
    Bt[n + e] = __float2bfloat16_rn(a - __bfloat162float(hi));
  }
}

struct RankList {
  int n;
  int R[kMaxModes];
};

// scal[0] = fitness, scal[1] = ||G||^2, scal[2 + 2n] = ||dA^(n)||^2,
// scal[3 + 2n] = ||A^(n)||^2 (sums of the per-column parts)
__global__ void tucker_scalars_kernel(const double* __restrict__ G, int64_t ng, double normX2,
                                      const double* __restrict__ part, RankList rl,
                                      double* __restrict__ scal) {
  __shared__ double red[256];
  double g = 0.0;
  for (int64_t i = threadIdx.x; i < ng; i += blockDim.x) g = fma(G[i], G[i], g);
  red[threadIdx.x] = g;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double gn = red[0];
    scal[0] = 1.0 - sqrt(fmax(normX2 - gn, 0.0)) / sqrt(normX2);
    scal[1] = gn;
    for (int n = 0; n < rl.n; n++) {
      double nd = 0.0, na = 0.0;
      for (int r = 0; r < rl.R[n]; r++) {
        nd += part[2 * (kTuckerMaxRank * n + r)];
        na += part[2 * (kTuckerMaxRank * n + r) + 1];
      }
      scal[2 + 2 * n] = nd;
      scal[3 + 2 * n] = na;
    }
  }
}

}  // namespace
}  // namespace cpals

using namespace cpals;

struct cpals_tucker {
  int N = 3;
  int64_t s[kMaxModes] = {};
  int R[kMaxModes] = {};
  int iters = 8;                       // subspace iterations per factor update
  cudaStream_t stream = nullptr;
  int64_t launches = 0;
  std::string err;
  double* X = nullptr;
  double normX2 = 0.0;
  bool have_tensor = false, have_factors = false, ops_built = false;
  double* A[kMaxModes] = {};
  double* Ap[kMaxModes] = {};
  double* dA[kMaxModes] = {};
  double *T = nullptr, *U = nullptr, *Y = nullptr, *Yt = nullptr, *G = nullptr;
  double *W = nullptr, *Z = nullptr, *Q = nullptr, *C = nullptr, *V = nullptr, *lam = nullptr;
  double* part = nullptr;              // kMaxModes * kTuckerMaxRank * 2 column norms
  double* C2 = nullptr;                // partial Grams of the convergence test
  double* rpart = nullptr;             // per-CTA residual sums
  double* gpart = nullptr;             // K-split partial sums of the contractions
  int64_t gpart_cap = 0;
  double* ops[kMaxModes * (kMaxModes - 1) / 2] = {};   // pairs i < n in lexicographic order
  double* Mp[kMaxModes] = {};
  // order N > 3: intermediates of the contraction chains (each up to the
  // largest single-mode contraction of X)
  double *Pa = nullptr, *Pb = nullptr, *Ya = nullptr, *Yb = nullptr;
  double* scal = nullptr;
  double* scal_h = nullptr;
  // tensor-core first level (CPALS_MIXED_BF16)
  bool mixed = false;
  __nv_bfloat16* Xb = nullptr;
  __nv_bfloat16* Bt = nullptr;
  float* outf = nullptr;
  float* gpartf = nullptr;
  int64_t gpartf_cap = 0;
  int* umma_sched = nullptr;
  int* status = nullptr;
  int status_h[2] = {0, 0};             // Cholesky-QR pivot bits, tensor-core kernel error
  Launch L() { return Launch{stream, &launches}; }
  cpals_status fail(cpals_status st, const std::string& m) {
    err = m;
    return st;
  }
};

namespace {

#define TK(x)                                                                  \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) return t->fail(CPALS_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define TKS(x)                                                                 \
  do {                                                                         \
    cpals_status s_ = (x);                                                     \
    if (s_ != CPALS_OK) return s_;                                             \
  } while (0)

// out = in x_mode B for the layouts of the file comment (gemm_simt: K-major
// contracts the trailing index, MN-major a leading or middle one); K is split
// so that the grid covers the SMs at least twice.  Batched MN-major calls
// with M, R <= 48 take bsmall_kernel: the rank-kept second-level TTMs and PP
// terms, and also a first-level TTM of X whose trailing mode is at most 48
// (exact outputs, no padded FMAs, one CTA per batch entry).
void gemm(cpals_tucker* t, const double* in, const double* B, double* out, int64_t batch, int64_t K,
          int64_t M, int R, bool kmajor) {
  if (!kmajor && batch > 1 && M <= kTuckerMaxRank && R <= kTuckerMaxRank && batch < (1ll << 31) &&
      K < (1ll << 31)) {
    bsmall_kernel<<<(unsigned)batch, 256, 0, t->stream>>>(in, B, (int)K, (int)M, R, out);
    t->launches++;
    return;
  }
  const int sp = gemm_simt_splits(batch, K, M, R, kmajor, t->gpart_cap, 2 * 152);
  gemm_simt<double, double>(in, B, out, t->gpart, batch, K, M, R, kmajor, sp, t->L());
}

// First-level TTM of X with factor A (K x R): out = X x_mode A in the layouts
// of gemm_simt; on the tensor cores in mixed precision.
cpals_status first_level(cpals_tucker* t, const double* A, double* out, int64_t batch, int64_t K,
                         int64_t M, int R, bool kmajor) {
  if (!t->mixed) {
    gemm(t, t->X, A, out, batch, K, M, R, kmajor);
    return CPALS_OK;
  }
  const int Rpad = (int)cdivt(R, 16) * 16;
  const int64_t Kstride = cdivt(K, 8) * 8;
  factor_bt_kernel<<<(unsigned)std::min<int64_t>(cdivt((int64_t)Rpad * Kstride, 256), 1216), 256, 0,
                     t->stream>>>(A, K, R, Rpad, Kstride, t->Bt);
  t->launches++;
  const int64_t mtiles = cdivt(M, 128) * batch;
  int splits = 1;
  if (mtiles < 2 * 152)
    splits = (int)std::max<int64_t>(1, std::min<int64_t>(cdivt(2 * 152, mtiles), cdivt(K, 256)));
  while (splits > 1 && (int64_t)splits * batch * M * R > t->gpartf_cap) splits--;
  TK(umma_gemm_bf16(t->Xb, t->Bt, t->outf, t->gpartf, batch, K, M, R, Rpad, Kstride, kmajor, splits,
                    t->status + 1, t->umma_sched, t->L()));
  convert<float, double>(t->outf, out, batch * M * R, t->L());
  return CPALS_OK;
}

// nb partial Grams of P^T Q (s rows of R) into dst (skipped once *skip is set)
int atb_parts(cpals_tucker* t, const double* P, const double* Q, int s, int R, double* dst,
              const int* skip) {
  const int rpb = (int)std::max<int64_t>(32, cdivt(cdivt(s, 128), 32) * 32);
  const int nb = (int)cdivt(s, rpb);
  atb_part_kernel<<<(unsigned)nb, 256, 0, t->stream>>>(P, Q, s, R, rpb, dst, skip);
  t->launches++;
  return nb;
}

// Leading R_n eigenvectors of W = Y_(n) Y_(n)^T into A[n] (Y: s_n rows of K)
cpals_status eig_update(cpals_tucker* t, int n, const double* Yn, int64_t K, const double* Aref) {
  const int s = (int)t->s[n], R = t->R[n];
  const unsigned tiles = (unsigned)cdivt(s, 16);
  syrk_kernel<<<dim3(tiles, tiles), 256, 0, t->stream>>>(Yn, s, (int)K, t->W);
  t->launches++;
  const unsigned rows_grid = (unsigned)std::min<int64_t>(cdivt(s, 8), 152);
  int* done = t->status + 2;
  TK(cudaMemsetAsync(done, 0, sizeof(int), t->stream));
  auto cholqr = [&](const double* in, const int* skip) {
    const int nb = atb_parts(t, in, in, s, R, t->C, skip);
    cholqr_kernel<<<rows_grid, 256, 0, t->stream>>>(t->C, nb, in, s, R, t->Q, t->status, skip);
    t->launches++;
  };
  // subspace iteration from the current factor: Z = W Q, orthonormalised by
  // Cholesky QR.  From the second step on, the invariance residual of the
  // current basis is tested first; once it is below 1e-13 the remaining steps
  // return at entry (no host round trip).  A last Cholesky QR pass always runs.
  const double* src = t->A[n];
  for (int it = 0; it < t->iters; it++) {
    const int* skip = it ? done : nullptr;
    rowmm_kernel<<<(unsigned)s, 256, 0, t->stream>>>(t->W, src, s, R, t->Z, skip);
    t->launches++;
    if (it) {
      const int nb2 = atb_parts(t, src, t->Z, s, R, t->C2, skip);
      resid_kernel<<<rows_grid, 256, 0, t->stream>>>(t->C2, nb2, src, t->Z, s, R, 1e-26, t->rpart,
                                                     t->status + 3, done);
      t->launches++;
    }
    cholqr(t->Z, skip);
    src = t->Q;
  }
  cholqr(t->Q, nullptr);
  // Rayleigh-Ritz: H = Q^T W Q, its eigenvectors V, A = Q V
  rowmm_kernel<<<(unsigned)s, 256, 0, t->stream>>>(t->W, t->Q, s, R, t->Z, nullptr);
  t->launches++;
  const int nb = atb_parts(t, t->Q, t->Z, s, R, t->C, nullptr);
  jacobi_kernel<<<1, 256, 0, t->stream>>>(t->C, nb, R, t->V, t->lam);
  qv_sign_kernel<<<(unsigned)R, 256, 0, t->stream>>>(t->Q, t->V, s, R, t->A[n], Aref, t->dA[n],
                                                    t->part + 2 * kTuckerMaxRank * n);
  t->launches += 2;
  return CPALS_OK;
}

// Y: Y^(N-1) as [x_{N-1}][r_0 .. r_{N-2}]
cpals_status finish_sweep(cpals_tucker* t, const double* Y) {
  // G = Y x_{N-1} A^(N-1): out[m = (r_0 .. r_{N-2})][r_{N-1}] = sum_x Y[x][m] A[x][r]
  const int N = t->N;
  int64_t m = 1;
  for (int k = 0; k + 1 < N; k++) m *= t->R[k];
  gemm(t, Y, t->A[N - 1], t->G, 1, t->s[N - 1], m, t->R[N - 1], false);
  RankList rl;
  rl.n = N;
  for (int k = 0; k < kMaxModes; k++) rl.R[k] = k < N ? t->R[k] : 0;
  tucker_scalars_kernel<<<1, 256, 0, t->stream>>>(t->G, m * t->R[N - 1], t->normX2, t->part, rl, t->scal);
  t->launches += 1;
  TK(cudaMemcpyAsync(t->scal_h, t->scal, (2 + 2 * N) * 8, cudaMemcpyDeviceToHost, t->stream));
  TK(cudaMemcpyAsync(t->status_h, t->status, 8, cudaMemcpyDeviceToHost, t->stream));
  TK(cudaStreamSynchronize(t->stream));
  TK(cudaGetLastError());
  if (t->status_h[1]) {
    TK(cudaMemset(t->status, 0, 8));
    return t->fail(CPALS_E_TIMEOUT, "tensor-core contraction gave up waiting (code " +
                                        std::to_string(t->status_h[1]) + ")");
  }
  if (t->status_h[0]) {
    TK(cudaMemset(t->status, 0, 8));
    return t->fail(CPALS_E_SINGULAR, "Cholesky QR met a non-positive pivot");
  }
  return CPALS_OK;
}

cpals_status tucker_als(cpals_tucker* t) {
  const int64_t s1 = t->s[0], s2 = t->s[1], s3 = t->s[2];
  const int R1 = t->R[0], R2 = t->R[1], R3 = t->R[2];
  // T = X x_3 A3 [x1][x2][r3]
  TKS(first_level(t, t->A[2], t->T, 1, s3, s1 * s2, R3, true));
  // Y1 = T x_2 A2 [x1][r3][r2]
  gemm(t, t->T, t->A[1], t->Y, s1, s2, R3, R2, false);
  TKS(eig_update(t, 0, t->Y, (int64_t)R3 * R2, nullptr));
  // Y2 = T x_1 A1 [x2][r3][r1]
  gemm(t, t->T, t->A[0], t->Y, 1, s1, s2 * R3, R1, false);
  TKS(eig_update(t, 1, t->Y, (int64_t)R3 * R1, nullptr));
  // U = X x_1 A1 [x2][x3][r1]; Y3 = U x_2 A2 [x3][r1][r2]
  TKS(first_level(t, t->A[0], t->U, 1, s1, s2 * s3, R1, false));
  gemm(t, t->U, t->A[1], t->Y, 1, s2, s3 * R1, R2, false);
  TKS(eig_update(t, 2, t->Y, (int64_t)R1 * R2, nullptr));
  return finish_sweep(t, t->Y);
}

cpals_status tucker_build(cpals_tucker* t) {
  const int64_t s1 = t->s[0], s2 = t->s[1], s3 = t->s[2];
  const int R1 = t->R[0], R2 = t->R[1], R3 = t->R[2];
  for (int n = 0; n < 3; n++)
    TK(cudaMemcpyAsync(t->Ap[n], t->A[n], t->s[n] * t->R[n] * 8, cudaMemcpyDeviceToDevice, t->stream));
  // Y_p^(1,2) = X x_3 A3 [x1][x2][r3]; Y_p^(1,3) = X x_2 A2 [x1][x3][r2]; Y_p^(2,3) = X x_1 A1 [x2][x3][r1]
  TKS(first_level(t, t->Ap[2], t->ops[0], 1, s3, s1 * s2, R3, true));
  TKS(first_level(t, t->Ap[1], t->ops[1], s1, s2, s3, R2, false));
  TKS(first_level(t, t->Ap[0], t->ops[2], 1, s1, s2 * s3, R1, false));
  // Y_p^(1) [x1][r3][r2], Y_p^(2) [x2][r3][r1], Y_p^(3) [x3][r1][r2]
  gemm(t, t->ops[0], t->Ap[1], t->Mp[0], s1, s2, R3, R2, false);
  gemm(t, t->ops[0], t->Ap[0], t->Mp[1], 1, s1, s2 * R3, R1, false);
  gemm(t, t->ops[2], t->Ap[1], t->Mp[2], 1, s2, s3 * R1, R2, false);
  for (int n = 0; n < 3; n++) TK(cudaMemsetAsync(t->dA[n], 0, t->s[n] * t->R[n] * 8, t->stream));
  t->ops_built = true;
  return CPALS_OK;
}

cpals_status tucker_pp(cpals_tucker* t) {
  const int64_t s1 = t->s[0], s2 = t->s[1], s3 = t->s[2];
  const int R1 = t->R[0], R2 = t->R[1], R3 = t->R[2];
  auto copy = [&](const double* in, double* out, int64_t n) {
    axpy_kernel<<<(unsigned)std::min<int64_t>(cdivt(n, 256), 1216), 256, 0, t->stream>>>(in, out, n, 0);
    t->launches++;
  };
  auto add = [&](const double* in, double* out, int64_t n) {
    axpy_kernel<<<(unsigned)std::min<int64_t>(cdivt(n, 256), 1216), 256, 0, t->stream>>>(in, out, n, 1);
    t->launches++;
  };
  auto addT = [&](const double* in, double* out, int64_t B, int P, int Qd) {
    add_transposed_kernel<<<(unsigned)std::min<int64_t>(cdivt(B * P * Qd, 256), 1216), 256, 0, t->stream>>>(
        in, out, B, P, Qd);
    t->launches++;
  };
  // mode 1: Y~1 [x1][r3][r2] = Mp1 + Y_p^(1,2) x_2 dA2 + Y_p^(1,3) x_3 dA3
  copy(t->Mp[0], t->Y, s1 * R3 * R2);
  gemm(t, t->ops[0], t->dA[1], t->Yt, s1, s2, R3, R2, false);            // [x1][r3][r2]
  add(t->Yt, t->Y, s1 * R3 * R2);
  gemm(t, t->ops[1], t->dA[2], t->Yt, s1, s3, R2, R3, false);            // [x1][r2][r3]
  addT(t->Yt, t->Y, s1, R3, R2);
  TKS(eig_update(t, 0, t->Y, (int64_t)R3 * R2, t->Ap[0]));
  // mode 2: Y~2 [x2][r3][r1] = Mp2 + Y_p^(1,2) x_1 dA1 + Y_p^(2,3) x_3 dA3
  copy(t->Mp[1], t->Y, s2 * R3 * R1);
  gemm(t, t->ops[0], t->dA[0], t->Yt, 1, s1, s2 * R3, R1, false);        // [x2][r3][r1]
  add(t->Yt, t->Y, s2 * R3 * R1);
  gemm(t, t->ops[2], t->dA[2], t->Yt, s2, s3, R1, R3, false);            // [x2][r1][r3]
  addT(t->Yt, t->Y, s2, R3, R1);
  TKS(eig_update(t, 1, t->Y, (int64_t)R3 * R1, t->Ap[1]));
  // mode 3: Y~3 [x3][r1][r2] = Mp3 + Y_p^(1,3) x_1 dA1 + Y_p^(2,3) x_2 dA2
  copy(t->Mp[2], t->Y, s3 * R1 * R2);
  gemm(t, t->ops[1], t->dA[0], t->Yt, 1, s1, s3 * R2, R1, false);        // [x3][r2][r1]
  addT(t->Yt, t->Y, s3, R1, R2);
  gemm(t, t->ops[2], t->dA[1], t->Yt, 1, s2, s3 * R1, R2, false);        // [x3][r1][r2]
  add(t->Yt, t->Y, s3 * R1 * R2);
  TKS(eig_update(t, 2, t->Y, (int64_t)R1 * R2, t->Ap[2]));
  return finish_sweep(t, t->Y);
}

// ---------------------------------------------------------------- order N > 3
// Tensors in these chains are row-major over a layout: the modes still at
// full size in increasing order, then the rank indices of the contracted
// modes in the order they were contracted.  Contracting the full mode at
// position p with A (s x R) is one gemm (batch = sizes before p, K = s, M =
// sizes after p, K-major when p is last) and appends that mode's rank index;
// contracting modes in increasing order therefore leaves the ranks in
// increasing mode order.  Canonical layouts: Y^(n) [x_n][r_k, k != n];
// operators Y_p^(i,n), i < n, [x_i][x_n][r_k, k not in {i, n}]; the core
// [r_0 .. r_{N-1}].
struct Layout {
  int n = 0;
  int mode[kMaxModes];
  bool rank[kMaxModes];
};

Layout full_layout(const cpals_tucker* t) {
  Layout l;
  l.n = t->N;
  for (int k = 0; k < t->N; k++) {
    l.mode[k] = k;
    l.rank[k] = false;
  }
  return l;
}

int64_t entry_size(const cpals_tucker* t, const Layout& l, int p) {
  return l.rank[p] ? t->R[l.mode[p]] : t->s[l.mode[p]];
}

// out = in x_j A (A: s_j x R_j); returns the new layout
Layout ttm_step(cpals_tucker* t, const double* in, const Layout& l, int j, const double* A, double* out) {
  int p = -1;
  for (int q = 0; q < l.n; q++)
    if (l.mode[q] == j && !l.rank[q]) p = q;
  int64_t pre = 1, post = 1;
  for (int q = 0; q < p; q++) pre *= entry_size(t, l, q);
  for (int q = p + 1; q < l.n; q++) post *= entry_size(t, l, q);
  if (post == 1) gemm(t, in, A, out, 1, t->s[j], pre, t->R[j], true);
  else gemm(t, in, A, out, pre, t->s[j], post, t->R[j], false);
  Layout o;
  o.n = 0;
  for (int q = 0; q < l.n; q++) {
    if (q == p) continue;
    o.mode[o.n] = l.mode[q];
    o.rank[o.n] = l.rank[q];
    o.n++;
  }
  o.mode[o.n] = j;
  o.rank[o.n] = true;
  o.n++;
  return o;
}

// src x_{k in modes} (in the given order) with factors F[k]; intermediates
// alternate between b0 and b1 (src is never written), the last step writes
// dst when given.  Returns the result's pointer.
const double* ttm_chain(cpals_tucker* t, const double* src, Layout& l, const int* modes, int nm,
                        double* const* F, double* b0, double* b1, double* dst) {
  const double* cur = src;
  for (int q = 0; q < nm; q++) {
    double* out = (q + 1 == nm && dst) ? dst : ((q & 1) ? b1 : b0);
    l = ttm_step(t, cur, l, modes[q], F[modes[q]], out);
    cur = out;
  }
  return cur;
}

int pair_index(int N, int i, int n) {   // i < n, lexicographic
  int idx = 0;
  for (int a = 0; a < i; a++) idx += N - 1 - a;
  return idx + (n - i - 1);
}

void permute_rank(cpals_tucker* t, const double* in, double* out, int n, int i, bool add) {
  // in [x_n][r_k, k not in {n, i}][r_i] -> out [x_n][r_k, k != n] (increasing k)
  int64_t a = 1, b = 1;
  for (int k = 0; k < t->N; k++) {
    if (k == n || k == i) continue;
    if (k < i) a *= t->R[k];
    else b *= t->R[k];
  }
  const int64_t total = t->s[n] * a * t->R[i] * b;
  permute_rank_kernel<<<(unsigned)std::min<int64_t>(cdivt(total, 256), 1216), 256, 0, t->stream>>>(
      in, out, t->s[n], a, t->R[i], b, add ? 1 : 0);
  t->launches++;
}

int64_t others_rank(const cpals_tucker* t, int n) {
  int64_t K = 1;
  for (int k = 0; k < t->N; k++)
    if (k != n) K *= t->R[k];
  return K;
}

Layout op_layout(const cpals_tucker* t, int i, int n) {   // Y_p^(i,n), i < n
  Layout l;
  l.n = 0;
  l.mode[l.n] = i;
  l.rank[l.n++] = false;
  l.mode[l.n] = n;
  l.rank[l.n++] = false;
  for (int k = 0; k < t->N; k++)
    if (k != i && k != n) {
      l.mode[l.n] = k;
      l.rank[l.n++] = true;
    }
  return l;
}

// HOOI sweep, order N: P_0 = X, P_{n+1} = P_n x_n A^(n) (the updated factor;
// [x_{n+1} .. x_{N-1}][r_0 .. r_n]) and Y^(n) = P_n x_{k > n} A^(k), so each
// sweep contracts X twice at full size (Y^(0)'s first step and P_1).
cpals_status tucker_als_n(cpals_tucker* t) {
  const int N = t->N;
  const double* P = t->X;
  Layout lp = full_layout(t);
  double* pbuf[2] = {t->Pa, t->Pb};
  int pi = 0;
  const double* Y = P;
  for (int n = 0; n < N; n++) {
    Y = P;
    if (n + 1 < N) {
      Layout ly = lp;
      int modes[kMaxModes], nm = 0;
      for (int k = n + 1; k < N; k++) modes[nm++] = k;
      Y = ttm_chain(t, P, ly, modes, nm, t->A, t->Ya, t->Yb, nullptr);
    }
    TKS(eig_update(t, n, Y, others_rank(t, n), nullptr));
    if (n + 1 < N) {
      double* out = pbuf[pi];
      pi ^= 1;
      lp = ttm_step(t, P, lp, n, t->A[n], out);
      P = out;
    }
  }
  return finish_sweep(t, Y);
}

// PP operators, order N (Sec. 3.2.2): Y_p^(i,n) = X x_{k not in {i,n}} A_p^(k)
// for every pair, grouped by the smallest contracted mode k0 (0, 1 or 2),
// whose contraction of X the group shares; then Y_p^(n) from one operator
// holding mode n; dA <- 0.
cpals_status tucker_build_n(cpals_tucker* t) {
  const int N = t->N;
  for (int n = 0; n < N; n++)
    TK(cudaMemcpyAsync(t->Ap[n], t->A[n], t->s[n] * t->R[n] * 8, cudaMemcpyDeviceToDevice, t->stream));
  for (int k0 = 0; k0 < 3; k0++) {
    bool first = true;
    Layout lt;
    for (int i = 0; i < N; i++)
      for (int n = i + 1; n < N; n++) {
        if (i == k0 || n == k0) continue;
        bool group = true;                 // every mode below k0 is kept
        for (int j = 0; j < k0; j++) group = group && (j == i || j == n);
        if (!group) continue;
        if (first) {
          lt = ttm_step(t, t->X, full_layout(t), k0, t->Ap[k0], t->Pa);
          first = false;
        }
        Layout l = lt;
        int modes[kMaxModes], nm = 0;
        for (int j = k0 + 1; j < N; j++)
          if (j != i && j != n) modes[nm++] = j;
        ttm_chain(t, t->Pa, l, modes, nm, t->Ap, t->Ya, t->Yb, t->ops[pair_index(N, i, n)]);
      }
  }
  for (int n = 0; n < N; n++) {
    const int i = n == 0 ? 1 : 0;
    const int lo = std::min(i, n), hi = std::max(i, n);
    ttm_step(t, t->ops[pair_index(N, lo, hi)], op_layout(t, lo, hi), i, t->Ap[i], t->Ya);
    permute_rank(t, t->Ya, t->Mp[n], n, i, false);
  }
  for (int n = 0; n < N; n++) TK(cudaMemsetAsync(t->dA[n], 0, t->s[n] * t->R[n] * 8, t->stream));
  t->ops_built = true;
  return CPALS_OK;
}

// PP sweep, order N: Y~^(n) = Y_p^(n) + sum_{i != n} Y_p^(i,n) x_i dA^(i)
// (Sec. 3.2.2) in the canonical layout, then the factor update as in ALS.
cpals_status tucker_pp_n(cpals_tucker* t) {
  const int N = t->N;
  for (int n = 0; n < N; n++) {
    const int64_t sz = t->s[n] * others_rank(t, n);
    axpy_kernel<<<(unsigned)std::min<int64_t>(cdivt(sz, 256), 1216), 256, 0, t->stream>>>(t->Mp[n], t->Pa, sz, 0);
    t->launches++;
    for (int i = 0; i < N; i++) {
      if (i == n) continue;
      const int lo = std::min(i, n), hi = std::max(i, n);
      ttm_step(t, t->ops[pair_index(N, lo, hi)], op_layout(t, lo, hi), i, t->dA[i], t->Ya);
      permute_rank(t, t->Ya, t->Pa, n, i, true);
    }
    TKS(eig_update(t, n, t->Pa, others_rank(t, n), t->Ap[n]));
  }
  return finish_sweep(t, t->Pa);
}

// Y^(N-1) at the current factors (the exact fitness), order N
const double* tucker_last_ttmc_n(cpals_tucker* t) {
  Layout l = full_layout(t);
  int modes[kMaxModes];
  for (int k = 0; k + 1 < t->N; k++) modes[k] = k;
  return ttm_chain(t, t->X, l, modes, t->N - 1, t->A, t->Pa, t->Pb, nullptr);
}

cpals_status run_als(cpals_tucker* t) { return t->N == 3 ? tucker_als(t) : tucker_als_n(t); }
cpals_status run_build(cpals_tucker* t) { return t->N == 3 ? tucker_build(t) : tucker_build_n(t); }
cpals_status run_pp(cpals_tucker* t) { return t->N == 3 ? tucker_pp(t) : tucker_pp_n(t); }

int64_t prod_dims(const cpals_tucker* t) {
  int64_t n = 1;
  for (int k = 0; k < t->N; k++) n *= t->s[k];
  return n;
}

cpals_status tk_ready(cpals_tucker* t) {
  if (!t) return CPALS_E_INVALID;
  if (!t->have_tensor) return t->fail(CPALS_E_STATE, "no tensor");
  if (!t->have_factors) return t->fail(CPALS_E_STATE, "no factors");
  return CPALS_OK;
}

}  // namespace

extern "C" {

cpals_status cpals_tucker_create(const int64_t* dims, int N, const int* ranks, cpals_tucker** out) {
  if (!out) return CPALS_E_INVALID;
  *out = nullptr;
  if (!dims || !ranks || N < 3 || N > kMaxModes) return CPALS_E_INVALID;
  for (int n = 0; n < N; n++)
    if (dims[n] < 1 || dims[n] > 4096 || ranks[n] < 1 || ranks[n] > kTuckerMaxRank || ranks[n] > dims[n])
      return CPALS_E_INVALID;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return CPALS_E_CUDA;
  }
  if (!(prop.major == 10 && prop.minor == 3)) return CPALS_E_UNSUPPORTED;
  cpals_tucker* t = new cpals_tucker();
  t->N = N;
  int64_t nx = 1, smax = 1, nr = 1;
  for (int n = 0; n < N; n++) {
    t->s[n] = dims[n];
    t->R[n] = ranks[n];
    nx *= dims[n];
    nr *= ranks[n];
    smax = std::max<int64_t>(smax, dims[n]);
  }
  // the largest single-mode contraction of X (order N: every chain
  // intermediate, operator and Y^(n) is at most this size)
  int64_t inter = 0;
  for (int n = 0; n < N; n++) inter = std::max<int64_t>(inter, nx / dims[n] * ranks[n]);
  const int64_t s1 = dims[0], s2 = dims[1], s3 = dims[2];
  const int R1 = ranks[0], R2 = ranks[1], R3 = ranks[2];
  const int64_t Ymax = N == 3 ? std::max(s1 * R2 * R3, std::max(s2 * R1 * R3, s3 * R1 * R2)) : inter;
  bool ok = cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking) == cudaSuccess;
  auto al = [&](double** p, int64_t n) {
    if (ok) ok = cudaMalloc((void**)p, (size_t)std::max<int64_t>(n, 1) * 8) == cudaSuccess;
  };
  al(&t->X, nx);
  for (int n = 0; n < N; n++) {
    al(&t->A[n], dims[n] * ranks[n]);
    al(&t->Ap[n], dims[n] * ranks[n]);
    al(&t->dA[n], dims[n] * ranks[n]);
  }
  if (N == 3) {
    al(&t->T, s1 * s2 * R3);
    al(&t->U, s2 * s3 * R1);
    al(&t->Y, Ymax);
    al(&t->Yt, Ymax);
  } else {
    al(&t->Pa, inter);
    al(&t->Pb, inter);
    al(&t->Ya, inter);
    al(&t->Yb, inter);
  }
  al(&t->G, nr);
  al(&t->W, smax * smax);
  al(&t->Z, smax * kTuckerMaxRank);
  al(&t->Q, smax * kTuckerMaxRank);
  al(&t->C, 128 * kTuckerMaxRank * kTuckerMaxRank);   // up to 128 partial Grams
  al(&t->C2, 128 * kTuckerMaxRank * kTuckerMaxRank);
  al(&t->rpart, 2 * 152);
  t->gpart_cap = std::max<int64_t>(1 << 20, 4 * Ymax);
  al(&t->gpart, t->gpart_cap);
  al(&t->V, kTuckerMaxRank * kTuckerMaxRank);
  al(&t->lam, kTuckerMaxRank);
  al(&t->part, kMaxModes * 2 * kTuckerMaxRank);
  for (int i = 0; i < N; i++)
    for (int n = i + 1; n < N; n++) al(&t->ops[pair_index(N, i, n)], dims[i] * dims[n] * (nr / ranks[i] / ranks[n]));
  for (int n = 0; n < N; n++) al(&t->Mp[n], dims[n] * (nr / ranks[n]));
  al(&t->scal, 32);
  if (ok) ok = cudaMalloc((void**)&t->status, 16) == cudaSuccess && cudaMemset(t->status, 0, 16) == cudaSuccess;
  if (ok) ok = cudaMallocHost((void**)&t->scal_h, 32 * 8) == cudaSuccess;
  if (ok) ok = cudaMemset(t->part, 0, kMaxModes * 2 * kTuckerMaxRank * 8) == cudaSuccess;
  if (ok) ok = setup_small_kernels() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cpals_tucker_destroy(t);
    return CPALS_E_OOM;
  }
  *out = t;
  return CPALS_OK;
}

void cpals_tucker_destroy(cpals_tucker* t) {
  if (!t) return;
  if (t->stream) cudaStreamSynchronize(t->stream);
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  F(t->X);
  for (int n = 0; n < kMaxModes; n++) {
    F(t->A[n]); F(t->Ap[n]); F(t->dA[n]); F(t->Mp[n]);
  }
  for (double* o : t->ops) F(o);
  F(t->T); F(t->U); F(t->Y); F(t->Yt); F(t->G); F(t->Pa); F(t->Pb); F(t->Ya); F(t->Yb); F(t->W); F(t->Z); F(t->Q); F(t->C); F(t->C2); F(t->rpart);
  F(t->V); F(t->lam); F(t->part); F(t->gpart); F(t->scal); F(t->status);
  F(t->Xb); F(t->Bt); F(t->outf); F(t->gpartf); F(t->umma_sched);
  if (t->scal_h) cudaFreeHost(t->scal_h);
  if (t->stream) cudaStreamDestroy(t->stream);
  cudaGetLastError();
  delete t;
}

cpals_status cpals_tucker_set_iterations(cpals_tucker* t, int iters) {
  if (!t || iters < 1 || iters > 1000) return CPALS_E_INVALID;
  t->iters = iters;
  return CPALS_OK;
}

cpals_status cpals_tucker_set_precision(cpals_tucker* t, int precision) {
  if (!t) return CPALS_E_INVALID;
  if (precision == CPALS_FP64) {
    t->mixed = false;
    return CPALS_OK;
  }
  if (precision != CPALS_MIXED_BF16) return t->fail(CPALS_E_INVALID, "precision must be FP64 or MIXED_BF16");
  if (t->N != 3) return t->fail(CPALS_E_UNSUPPORTED, "tensor-core TTMs: order 3 only");
  const int64_t s1 = t->s[0], s2 = t->s[1], s3 = t->s[2];
  if (!umma_supported(s3, s1 * s2, true, t->R[2]) || !umma_supported(s1, s2 * s3, false, t->R[0]) ||
      !umma_supported(s2, s3, false, t->R[1]))
    return t->fail(CPALS_E_UNSUPPORTED, "tensor-core TTM needs s_3 and s_2 s_3 multiples of 8");
  if (!t->Xb) {
    const int64_t n = s1 * s2 * s3;
    const int64_t kmax = cdivt(std::max(s1, std::max(s2, s3)), 8) * 8;
    const int64_t omax = std::max(s1 * s2 * t->R[2], std::max(s2 * s3 * t->R[0], s1 * s3 * t->R[1]));
    t->gpartf_cap = std::max<int64_t>(1 << 22, 2 * omax);
    bool ok = cudaMalloc((void**)&t->Xb, n * 2) == cudaSuccess &&
              cudaMalloc((void**)&t->Bt, 2 * 64 * kmax * 2) == cudaSuccess &&
              cudaMalloc((void**)&t->outf, omax * 4) == cudaSuccess &&
              cudaMalloc((void**)&t->gpartf, t->gpartf_cap * 4) == cudaSuccess &&
              cudaMalloc((void**)&t->umma_sched, 2 * sizeof(int)) == cudaSuccess &&
              cudaMemset(t->umma_sched, 0, 2 * sizeof(int)) == cudaSuccess &&
              setup_umma_kernels() == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      auto F = [](void* p) { if (p) cudaFree(p); };
      F(t->Xb); F(t->Bt); F(t->outf); F(t->gpartf); F(t->umma_sched);
      t->Xb = nullptr; t->Bt = nullptr; t->outf = nullptr; t->gpartf = nullptr; t->umma_sched = nullptr;
      return t->fail(CPALS_E_OOM, "tensor-core buffers");
    }
  }
  t->mixed = true;
  if (t->have_tensor) {
    to_bf16_kernel<<<1216, 256, 0, t->stream>>>(t->X, t->Xb, t->s[0] * t->s[1] * t->s[2]);
    t->launches++;
    TK(cudaStreamSynchronize(t->stream));
    TK(cudaGetLastError());
  }
  t->ops_built = false;
  return CPALS_OK;
}

cpals_status cpals_tucker_set_tensor(cpals_tucker* t, const void* data, int dtype, int on_device) {
  if (!t || !data || (dtype != 0 && dtype != 1)) return t ? t->fail(CPALS_E_INVALID, "bad tensor") : CPALS_E_INVALID;
  const int64_t n = prod_dims(t);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (dtype == 0) {
    TK(cudaMemcpyAsync(t->X, data, n * 8, kind, t->stream));
  } else {
    float* tmp = nullptr;
    TK(cudaMalloc((void**)&tmp, n * 4));
    cudaError_t e = cudaMemcpyAsync(tmp, data, n * 4, kind, t->stream);
    if (e == cudaSuccess) {
      convert<float, double>(tmp, t->X, n, t->L());
      e = cudaStreamSynchronize(t->stream);
    }
    cudaFree(tmp);
    TK(e);
  }
  sumsq<double>(t->X, n, t->gpart, t->scal + 31, t->L());
  TK(cudaMemcpyAsync(t->scal_h + 31, t->scal + 31, 8, cudaMemcpyDeviceToHost, t->stream));
  TK(cudaStreamSynchronize(t->stream));
  TK(cudaGetLastError());
  t->normX2 = t->scal_h[31];
  if (t->mixed) {
    to_bf16_kernel<<<1216, 256, 0, t->stream>>>(t->X, t->Xb, n);
    t->launches++;
    TK(cudaStreamSynchronize(t->stream));
    TK(cudaGetLastError());
  }
  t->have_tensor = true;
  t->ops_built = false;
  return CPALS_OK;
}

cpals_status cpals_tucker_init_factors(cpals_tucker* t, const double* const* factors) {
  if (!t || !factors) return t ? t->fail(CPALS_E_INVALID, "factors is NULL") : CPALS_E_INVALID;
  for (int n = 0; n < t->N; n++) {
    if (!factors[n]) return t->fail(CPALS_E_INVALID, "factor pointer is NULL");
    TK(cudaMemcpyAsync(t->A[n], factors[n], t->s[n] * t->R[n] * 8, cudaMemcpyHostToDevice, t->stream));
    // Algorithm 4 starts from dA <- A
    TK(cudaMemcpyAsync(t->dA[n], t->A[n], t->s[n] * t->R[n] * 8, cudaMemcpyDeviceToDevice, t->stream));
  }
  TK(cudaStreamSynchronize(t->stream));
  for (int n = 0; n < t->N; n++) {
    t->scal_h[2 + 2 * n] = t->R[n];       // ||dA||^2 = ||A||^2 = R for orthonormal columns
    t->scal_h[3 + 2 * n] = t->R[n];
  }
  t->have_factors = true;
  t->ops_built = false;
  return CPALS_OK;
}

cpals_status cpals_tucker_als_sweep(cpals_tucker* t, double* fitness) {
  TKS(tk_ready(t));
  TKS(run_als(t));
  if (fitness) *fitness = t->scal_h[0];
  return CPALS_OK;
}

cpals_status cpals_tucker_pp_build_operators(cpals_tucker* t) {
  TKS(tk_ready(t));
  TKS(run_build(t));
  TK(cudaStreamSynchronize(t->stream));
  TK(cudaGetLastError());
  return CPALS_OK;
}

cpals_status cpals_tucker_pp_sweep(cpals_tucker* t, double* fitness) {
  TKS(tk_ready(t));
  if (!t->ops_built) return t->fail(CPALS_E_STATE, "PP operators not built");
  TKS(run_pp(t));
  if (fitness) *fitness = t->scal_h[0];
  return CPALS_OK;
}

cpals_status cpals_tucker_run(cpals_tucker* t, int max_sweeps, double eps, double* fitness_trace,
                              int* kind_trace, int* n_done) {
  TKS(tk_ready(t));
  if (max_sweeps < 0) return t->fail(CPALS_E_INVALID, "max_sweeps < 0");
  auto small = [&]() {
    for (int n = 0; n < t->N; n++)
      if (!(t->scal_h[2 + 2 * n] < eps * eps * t->scal_h[3 + 2 * n])) return false;
    return true;
  };
  int k = 0;
  cpals_status st = CPALS_OK;
  auto record = [&](int kind) {
    if (fitness_trace) fitness_trace[k] = t->scal_h[0];
    if (kind_trace) kind_trace[k] = kind;
    k++;
  };
  while (st == CPALS_OK && k < max_sweeps) {
    if (eps > 0 && small()) {
      st = run_build(t);
      if (st != CPALS_OK) break;
      // dA <- 0 after the operators are formed (Algorithm 4)
      for (int n = 0; n < t->N; n++) t->scal_h[2 + 2 * n] = 0.0;
      bool first = true;
      while (st == CPALS_OK && k < max_sweeps && small()) {
        st = run_pp(t);
        if (st != CPALS_OK) break;
        record(first ? CPALS_SWEEP_PP_INIT : CPALS_SWEEP_PP_APPROX);
        first = false;
      }
      if (st != CPALS_OK || k >= max_sweeps) break;
    }
    st = run_als(t);
    if (st != CPALS_OK) break;
    record(CPALS_SWEEP_ALS);
  }
  if (n_done) *n_done = k;
  return st;
}

cpals_status cpals_tucker_fitness(cpals_tucker* t, double* out) {
  TKS(tk_ready(t));
  if (!out) return t->fail(CPALS_E_INVALID, "out is NULL");
  // exact: Y^(N-1) and the core at the current factors
  if (t->N == 3) {
    const int64_t s1 = t->s[0], s2 = t->s[1], s3 = t->s[2];
    TKS(first_level(t, t->A[0], t->U, 1, s1, s2 * s3, t->R[0], false));
    gemm(t, t->U, t->A[1], t->Yt, 1, s2, s3 * t->R[0], t->R[1], false);
    TKS(finish_sweep(t, t->Yt));
  } else {
    TKS(finish_sweep(t, tucker_last_ttmc_n(t)));
  }
  *out = t->scal_h[0];
  return CPALS_OK;
}

cpals_status cpals_tucker_get_factors(cpals_tucker* t, double* const* out) {
  if (!t || !out) return CPALS_E_INVALID;
  for (int n = 0; n < t->N; n++) {
    if (!out[n]) return t->fail(CPALS_E_INVALID, "NULL buffer");
    TK(cudaMemcpyAsync(out[n], t->A[n], t->s[n] * t->R[n] * 8, cudaMemcpyDeviceToHost, t->stream));
  }
  TK(cudaStreamSynchronize(t->stream));
  return CPALS_OK;
}

cpals_status cpals_tucker_get_core(cpals_tucker* t, double* out) {
  if (!t || !out) return CPALS_E_INVALID;
  int64_t nr = 1;
  for (int n = 0; n < t->N; n++) nr *= t->R[n];
  TK(cudaMemcpyAsync(out, t->G, (size_t)nr * 8, cudaMemcpyDeviceToHost, t->stream));
  TK(cudaStreamSynchronize(t->stream));
  return CPALS_OK;
}

const char* cpals_tucker_last_error(const cpals_tucker* t) { return t ? t->err.c_str() : "null context"; }

cpals_status cpals_tucker_cost_model(const int64_t* dims, const int* ranks, int kind, double* flops) {
  if (!dims || !ranks || !flops) return CPALS_E_INVALID;
  for (int n = 0; n < 3; n++)
    if (dims[n] < 1 || ranks[n] < 1) return CPALS_E_INVALID;
  const double s1 = (double)dims[0], s2 = (double)dims[1], s3 = (double)dims[2];
  const double R1 = ranks[0], R2 = ranks[1], R3 = ranks[2];
  const double X = s1 * s2 * s3;
  double f = 0.0;
  if (kind == 0) {
    // T = X x3 A3, Y1 = T x2 A2, Y2 = T x1 A1, U = X x1 A1, Y3 = U x2 A2, G = Y3 x3 A3
    f = 2 * X * R3 + 2 * s1 * s2 * R3 * R2 + 2 * s1 * s2 * R3 * R1 + 2 * X * R1 +
        2 * s2 * s3 * R1 * R2 + 2 * s3 * R1 * R2 * R3;
  } else if (kind == 1) {
    // three first-level operators, then Y_p^(1), Y_p^(2), Y_p^(3)
    f = 2 * X * (R1 + R2 + R3) + 2 * s1 * s2 * R3 * R2 + 2 * s1 * s2 * R3 * R1 +
        2 * s2 * s3 * R1 * R2;
  } else if (kind == 2) {
    // two first-order corrections per mode, then the core estimate
    f = 2 * s1 * s2 * R3 * R2 + 2 * s1 * s3 * R2 * R3 + 2 * s1 * s2 * R3 * R1 +
        2 * s2 * s3 * R1 * R3 + 2 * s1 * s3 * R2 * R1 + 2 * s2 * s3 * R1 * R2 +
        2 * s3 * R1 * R2 * R3;
  } else if (kind == 3) {
    // the paper's operator-construction sum for N = 3 (one level, l = 2):
    // 2 C(3,2) s^3 R, equidimensional
    if (dims[0] != dims[1] || dims[1] != dims[2] || ranks[0] != ranks[1] || ranks[1] != ranks[2])
      return CPALS_E_INVALID;
    f = 2.0 * 3.0 * X * R1;
  } else {
    return CPALS_E_INVALID;
  }
  *flops = f;
  return CPALS_OK;
}

}  // extern "C"
