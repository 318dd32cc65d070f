// Symmetric eigendecomposition by the cyclic Jacobi method, one CTA, for the
// pseudo-inverse Gamma^dagger that Algorithm 1 writes (Sec. 2.3) when Gamma is
// not positive definite.  Golub & Van Loan: the symmetric Schur 2 x 2
// rotation and the round-robin parallel ordering (R/2 disjoint rotations per
// round, R - 1 rounds per sweep), sweeps until the off-diagonal Frobenius
// norm is below 1e-15 of the total.  Shared by the float64 normal equations,
// the double-float ones and the fused batch.
#pragma once

#include <cuda_runtime.h>

namespace cpals {

constexpr int kJacobiSweeps = 30;
constexpr int kJacobiMaxRank = 128;

// G (R x R, row stride GS) becomes diag(w) = V^T G V; V (row stride VS) must
// hold the identity on entry and receives the eigenvectors as columns.  Every
// thread of the CTA calls it; G and V are read and written by all of them.
__device__ inline void sym_eig_jacobi(double* G, int GS, double* V, int VS, int R) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int RR = R * R;
  __shared__ double rc[kJacobiMaxRank / 2 + 1], rs_[kJacobiMaxRank / 2 + 1];
  __shared__ int rp[kJacobiMaxRank / 2 + 1], rq[kJacobiMaxRank / 2 + 1];
  __shared__ double red[2][32];
  const int m = R + (R & 1);                  // round-robin players (one idle when R is odd)
  for (int sweep = 0; sweep < kJacobiSweeps; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < RR; idx += nt) {
      const int i = idx / R, j = idx % R;
      const double v = G[i * GS + j];
      tot = fma(v, v, tot);
      if (i != j) off = fma(v, v, off);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (lane == 0) {
      red[0][warp] = off;
      red[1][warp] = tot;
    }
    __syncthreads();
    off = 0.0;
    tot = 0.0;
    for (int k = 0; k < nw; k++) {
      off += red[0][k];
      tot += red[1][k];
    }
    __syncthreads();                            // red is reused by the next sweep
    if (off <= 1e-30 * tot) break;
    for (int rd = 0; rd < m - 1; rd++) {
      for (int k = tid; k < m / 2; k += nt) {
        const int a = k == 0 ? m - 1 : (rd + k) % (m - 1);
        const int b = k == 0 ? rd : (rd - k + m - 1) % (m - 1);
        const int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < R) {
          const double apq = G[p * GS + q];
          if (apq != 0.0) {
            const double th = (G[q * GS + q] - G[p * GS + p]) / (2.0 * apq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(fma(th, th, 1.0)));
            c = 1.0 / sqrt(fma(t, t, 1.0));
            s = t * c;
          }
        }
        rp[k] = p;
        rq[k] = q;
        rc[k] = c;
        rs_[k] = s;
      }
      __syncthreads();
      // rows p and q of every pair: G <- J^T G
      for (int e = tid; e < (m / 2) * R; e += nt) {
        const int k = e / R, j = e % R;
        const double s = rs_[k];
        if (rq[k] >= R || s == 0.0) continue;
        const double c = rc[k];
        double* gp = G + rp[k] * GS + j;
        double* gq = G + rq[k] * GS + j;
        const double x = *gp, y = *gq;
        *gp = c * x - s * y;
        *gq = s * x + c * y;
      }
      __syncthreads();
      // columns p and q: G <- G J, V <- V J
      for (int e = tid; e < (m / 2) * R; e += nt) {
        const int k = e / R, i = e % R;
        const double s = rs_[k];
        if (rq[k] >= R || s == 0.0) continue;
        const double c = rc[k];
        const int p = rp[k], q = rq[k];
        const double x = G[i * GS + p], y = G[i * GS + q];
        G[i * GS + p] = c * x - s * y;
        G[i * GS + q] = s * x + c * y;
        const double vx = V[i * VS + p], vy = V[i * VS + q];
        V[i * VS + p] = c * vx - s * vy;
        V[i * VS + q] = s * vx + c * vy;
      }
      __syncthreads();
    }
  }
}

// The eigenvalues' pseudo-inverse weights into w (shared, R entries): for
// Gamma^dagger = V diag(w) V^T with pow = -1, or for the factor
// W = diag(w) V^T (Gamma^dagger = W^T W) with pow = -1/2; eigenvalues at or
// below 1e-13 of the largest get 0.
__device__ inline void pinv_weights(const double* G, int GS, int R, bool half, double* w) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < R; i += nt) w[i] = G[i * GS + i];
  __syncthreads();
  double wmax = 0.0;
  for (int i = 0; i < R; i++) wmax = fmax(wmax, w[i]);
  const double cut = 1e-13 * wmax;
  __syncthreads();
  for (int i = tid; i < R; i += nt) w[i] = w[i] > cut ? (half ? 1.0 / sqrt(w[i]) : 1.0 / w[i]) : 0.0;
  __syncthreads();
}

}  // namespace cpals
