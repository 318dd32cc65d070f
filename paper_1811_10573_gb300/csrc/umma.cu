// tcgen05 (5th-generation tensor core) first-level contraction for sm_103a.
//
// The first level of both dimension trees (Sec. 2.5, Sec. 3.2.3) contracts the
// input tensor X with one factor or with the Khatri-Rao product of a block of
// factors: a matrix product whose long dimension streams X from HBM once.
//   kmajor:  out[m][r]    = sum_k X[m*K + k]         * Bt[r][k]
//   !kmajor: out[b][m][r] = sum_k X[(b*K + k)*M + m] * Bt[r][k]
// X is bf16 (one-time copy of the input).  The B operand (a factor or a
// Khatri-Rao product, float32) is carried as two bf16 planes, Bt = hi + lo with
// hi = bf16(b) and lo = bf16(b - hi) (Rpad x Kstride each, zero padded).  The
// two planes sit one after the other in shared memory and enter one MMA as a
// B operand of 2 Rpad rows: the accumulator holds the hi products in columns
// [0, Rpad) and the lo products in [Rpad, 2 Rpad), which the epilogue adds.
// The factor thus enters with ~16 significant bits and only the one-time
// rounding of X remains (the same for every contraction path, which keeps
// the PP and ALS right-hand sides consistent).
//
// Persistent warp-specialised kernel, one CTA per SM.  A work unit is one or
// two 128-row output tiles (tpu) of one K chunk; the two tiles of a unit share
// every stage of the B operand, which halves the B traffic per byte of X and
// doubles the X bytes in flight.  The producer takes units from a global
// counter (atomicAdd) and passes each unit index to the MMA and epilogue
// warps through a four-slot queue in shared memory, so a CTA that starts
// late (its SM held by another kernel, e.g. the factorisation on the side
// stream) takes fewer units instead of finishing last; the last CTA to exit
// resets the counter for the next launch on the stream.
//   warp 0      : TMA producer (tpu A tiles 128 x 64 and the B tile 2 x Rpad x
//                 64 per stage, 128-byte swizzle, mbarrier complete_tx)
//   warp 1      : TMEM allocation + single-thread tcgen05.mma issue (M = 128,
//                 N = 2 Rpad, K = 16 per instruction), tcgen05.commit to free
//                 stages and to publish finished accumulators
//   warps 2..5  : epilogue: tcgen05.ld 32x32b into 128-byte-swizzled shared
//                 boxes of 128 rows x 32 columns (two, alternating), each
//                 written out by one TMA tensor store (R % 4 == 0), or a
//                 padded staging tile and coalesced row copies (otherwise)
// Each accumulator takes 256 TMEM columns (512 in all): with one tile per
// unit two accumulators let the epilogue of one unit run under the MMAs of
// the next; two tiles per unit are used only when every CTA has a single
// unit.  Every wait is bounded: on timeout the kernel records an error code,
// drains what it issued and returns.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace cpals {

namespace {

constexpr int BM = 128;
constexpr int BK = 64;                 // bf16 elements = 128 bytes = one swizzle row
constexpr int kThreadsUmma = 192;      // 6 warps
constexpr int A_STAGE_BYTES = BM * BK * 2;
// Default bound of the waits on work (a stage, an accumulator, the unit
// queue), ~2 s at 2 GHz; a launch may pass a shorter one (UmmaParams.wait_limit).
// The drain waits at exit (loads and MMAs already issued must land before the
// CTA releases shared memory and TMEM) always use this bound.
constexpr unsigned long long kTimeoutCycles = 4000000000ull;

// error codes written to the error word
enum { ERR_PRODUCER = 1, ERR_MMA_FULL = 2, ERR_MMA_ACC = 3, ERR_EPI = 4, ERR_DRAIN = 5 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait (limit in SM clock cycles); returns false on timeout or when
// another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          bool sleep, unsigned long long limit) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = clock64();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) return false;
    if (sleep) __nanosleep(64);
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, uint32_t src, int c0, int c1,
                                             int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(map),
      "r"(src), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 at [0,14), leading
// byte offset >> 4 at [16,30), stride byte offset >> 4 at [32,46), fixed
// 0b001 at [46,49), swizzle mode at [61,64) (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D fp32 (bits 4-5 = 1), A and B bf16
// (bits 7-9 = 1, 10-12 = 1), A major at bit 15 (1 = MN-major), B K-major,
// N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, bool a_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

struct UmmaParams {
  int64_t batch, K, M;
  int R, Rpad, splits, stages;
  int RS;               // row stride (floats) of the padded staging tile (no TMA store)
  int nbox;             // 32-column boxes of the swizzled staging tile (TMA store)
  int tma_store;        // 1: epilogue through TMA tensor stores
  int tpu;              // output tiles per unit (1 or 2)
  int64_t kchunk;       // multiple of BK
  int64_t mtiles, mgroups, units;
  float* out;           // out or partials ([z][b][m][r])
  int* err;
  int* sched;           // [next unit, CTAs done], zero at launch; null: static round robin
  unsigned long long wait_limit;   // bound of the waits on work, SM clock cycles
};

template <bool KMAJOR>
__global__ void __launch_bounds__(kThreadsUmma, 1)
umma_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 const __grid_constant__ CUtensorMap mapO, UmmaParams p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[8], empty_bar[8], accf_bar[2], acce_bar[2], done_bar;
  __shared__ __align__(8) uint64_t uq_full[4], uq_empty[4];   // unit queue
  __shared__ long long uq[4];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int S = p.stages;
  const int TPU = p.tpu;
  const uint32_t b_plane = (uint32_t)p.Rpad * BK * 2;
  const uint32_t b_stage_bytes = 2 * b_plane;
  const uint32_t a_bytes = (uint32_t)TPU * A_STAGE_BYTES;
  const uint32_t stage_bytes = a_bytes + b_stage_bytes;
  const uint32_t tmem_cols = 512;
  const int NBUF = TPU == 1 ? 2 : 1;            // accumulator sets (256 columns per tile)

  if (threadIdx.x == 0) {
    abort_sh = 0;
    for (int s = 0; s < S; s++) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(smem_u32(&accf_bar[b]), 1);
      mbar_init(smem_u32(&acce_bar[b]), 4);
    }
    mbar_init(smem_u32(&done_bar), 1);
    for (int q = 0; q < 4; q++) {
      mbar_init(smem_u32(&uq_full[q]), 1);
      mbar_init(smem_u32(&uq_empty[q]), 5);    // the MMA thread and the four epilogue warps
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapB) : "memory");
    if (p.tma_store) asm volatile("prefetch.tensormap [%0];" ::"l"(&mapO) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)), "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_sh;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      bool ok = true;
      for (int t = 0;; t++) {
        // next unit (-1 ends the queue); slot t % 4 is free once unit t-4 was read
        const int64_t un = p.sched ? (int64_t)atomicAdd(p.sched, 1)
                                   : (int64_t)blockIdx.x + (int64_t)t * gridDim.x;
        const int64_t u = (ok && un < p.units) ? un : -1;
        if (!mbar_wait(smem_u32(&uq_empty[t & 3]), ((t >> 2) & 1) ^ 1, &abort_sh, false, p.wait_limit)) {
          ok = false;
          break;
        }
        uq[t & 3] = u;
        mbar_arrive(smem_u32(&uq_full[t & 3]));
        if (u < 0) break;
        const int64_t mg = u % p.mgroups;
        const int64_t rest = u / p.mgroups;
        const int z = (int)(rest % p.splits);
        const int64_t b = rest / p.splits;
        const int64_t mt0 = mg * TPU;
        const int nt = (int)min((int64_t)TPU, p.mtiles - mt0);   // tiles in this unit
        const int64_t k0 = (int64_t)z * p.kchunk;
        const int64_t k1 = min(p.K, k0 + p.kchunk);
        for (int64_t k = k0; k < k1; k += BK) {
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, &abort_sh, false, p.wait_limit)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          const uint32_t sA = base + stage * stage_bytes;
          const uint32_t sB = sA + a_bytes;
          mbar_expect_tx(fb, (uint32_t)nt * A_STAGE_BYTES + b_stage_bytes);
          for (int tt = 0; tt < nt; tt++) {
            const uint32_t sAt = sA + tt * A_STAGE_BYTES;
            const int64_t mt = mt0 + tt;
            if (KMAJOR) {
              tma_load_2d(sAt, &mapA, fb, (int)k, (int)(mt * BM));
            } else {
              tma_load_3d(sAt, &mapA, fb, (int)(mt * BM), (int)k, (int)b);
              tma_load_3d(sAt + A_STAGE_BYTES / 2, &mapA, fb, (int)(mt * BM + 64), (int)k, (int)b);
            }
          }
          tma_load_3d(sB, &mapB, fb, (int)k, 0, 0);       // hi and lo planes
          issued[stage]++;
          if (++stage == S) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) {
          // the consumers may wait on this unit's stages: stop them
          atomicCAS(p.err, 0, ERR_PRODUCER);
          abort_sh = 1;
          break;
        }
      }
      if (!ok) {
        atomicCAS(p.err, 0, ERR_PRODUCER);
        abort_sh = 1;
      }
      // drain: every stage's last load has landed before the CTA may exit
      for (int s = 0; s < S; s++) {
        if (!issued[s]) continue;
        const uint32_t par = (uint32_t)((issued[s] - 1) & 1);
        const unsigned long long t0 = clock64();
        while (!mbar_try(smem_u32(&full_bar[s]), par)) {
          if (clock64() - t0 > kTimeoutCycles) {
            atomicCAS(p.err, 0, ERR_DRAIN);
            break;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc(BM, 2 * p.Rpad, !KMAJOR);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      bool any = false;
      for (int t = 0;; t++) {
        if (!mbar_wait(smem_u32(&uq_full[t & 3]), (t >> 2) & 1, &abort_sh, false, p.wait_limit)) {
          atomicCAS(p.err, 0, ERR_MMA_ACC);
          abort_sh = 1;
          break;
        }
        const int64_t u = uq[t & 3];
        mbar_arrive(smem_u32(&uq_empty[t & 3]));
        if (u < 0) break;
        const int64_t mg = u % p.mgroups;
        const int64_t rest = u / p.mgroups;
        const int z = (int)(rest % p.splits);
        const int nt = (int)min((int64_t)TPU, p.mtiles - mg * TPU);
        const int64_t k0 = (int64_t)z * p.kchunk;
        const int64_t k1 = min(p.K, k0 + p.kchunk);
        const int buf = t % NBUF;
        if (!mbar_wait(smem_u32(&acce_bar[buf]), ((t / NBUF) & 1) ^ 1, &abort_sh, false, p.wait_limit)) {
          atomicCAS(p.err, 0, ERR_MMA_ACC);
          abort_sh = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(buf * TPU * 256);
        uint32_t accum = 0;
        for (int64_t k = k0; k < k1; k += BK) {
          if (!mbar_wait(smem_u32(&full_bar[stage]), phase, &abort_sh, false, p.wait_limit)) {
            atomicCAS(p.err, 0, ERR_MMA_FULL);
            abort_sh = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sA = base + stage * stage_bytes;
          const uint32_t sB = sA + a_bytes;
#pragma unroll
          for (int ks = 0; ks < BK / 16; ks++) {
            // hi and lo planes: one B operand of 2 Rpad rows
            const uint64_t bdesc = smem_desc(sB + ks * 32, 16, 1024);
            for (int tt = 0; tt < nt; tt++) {
              const uint32_t sAt = sA + tt * A_STAGE_BYTES;
              uint64_t adesc;
              if (KMAJOR) adesc = smem_desc(sAt + ks * 32, 16, 1024);
              else adesc = smem_desc(sAt + ks * 2048, A_STAGE_BYTES / 2, 1024);
              umma_f16(d_tmem + (uint32_t)(tt * 256), adesc, bdesc, idesc, accum);
            }
            accum = 1;
          }
          umma_commit(smem_u32(&empty_bar[stage]));
          any = true;
          if (++stage == S) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        umma_commit(smem_u32(&accf_bar[buf]));
      }
      // all issued MMAs complete before TMEM is released
      if (any) {
        umma_commit(smem_u32(&done_bar));
        const unsigned long long t0 = clock64();
        while (!mbar_try(smem_u32(&done_bar), 0)) {
          if (clock64() - t0 > kTimeoutCycles) {
            atomicCAS(p.err, 0, ERR_DRAIN);
            break;
          }
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 2..5)
    // TMEM -> registers -> shared staging -> global.
    //  * TMA store path (R % 4 == 0): each 128-row x 32-column box is staged
    //    with the 128-byte swizzle (16-byte chunk c of row r at chunk
    //    c ^ (r % 8): conflict-free writes) in one of two alternating
    //    buffers and written by one tensor store; the tensor map's M extent
    //    clips the rows past the end of a batch and its R extent the padding
    //    columns.
    //  * otherwise: padded staging of the tile (row stride RS, RS/4 odd) and
    //    coalesced row copies.
    uint8_t* stg_base = smem_raw + (base - smem_u32(smem_raw)) + (size_t)S * stage_bytes;
    const uint32_t stg_u32 = base + S * stage_bytes;
    float* stg = reinterpret_cast<float*>(stg_base);
    const int q = warp & 3;                   // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    const int ew = warp - 2;
    const bool leader = (ew == 0 && lane == 0);
    int bc = 0;                               // boxes stored so far (alternating buffers)
    for (int t = 0;; t++) {
      long long uu = 0;
      int okq = 1;
      if (lane == 0) {
        okq = mbar_wait(smem_u32(&uq_full[t & 3]), (t >> 2) & 1, &abort_sh, true, p.wait_limit) ? 1 : 0;
        if (okq) {
          uu = uq[t & 3];
          mbar_arrive(smem_u32(&uq_empty[t & 3]));
        }
      }
      okq = __shfl_sync(0xffffffffu, okq, 0);
      if (!okq) {
        if (lane == 0) {
          atomicCAS(p.err, 0, ERR_EPI);
          abort_sh = 1;
        }
        break;
      }
      const int64_t u = (int64_t)__shfl_sync(0xffffffffu, uu, 0);
      if (u < 0) break;
      const int64_t mg = u % p.mgroups;
      const int64_t rest = u / p.mgroups;
      const int z = (int)(rest % p.splits);
      const int64_t b = rest / p.splits;
      const int nt = (int)min((int64_t)TPU, p.mtiles - mg * TPU);
      const int buf = t % NBUF;
      const uint32_t par = (uint32_t)((t / NBUF) & 1);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(smem_u32(&accf_bar[buf]), par, &abort_sh, true, p.wait_limit) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          atomicCAS(p.err, 0, ERR_EPI);
          abort_sh = 1;
        }
        break;
      }
      // the phase is complete for every lane once lane 0 has seen it
      while (!mbar_try(smem_u32(&accf_bar[buf]), par)) {
      }
      __syncwarp();
      tc_fence_after();
      const int zb = (int)((int64_t)z * p.batch + b);
      for (int tt = 0; tt < nt; tt++) {
        const int64_t m0 = (mg * TPU + tt) * BM;
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)((buf * TPU + tt) * 256);
        if (p.tma_store) {
          for (int bx = 0; bx < p.nbox; bx++, bc++) {
            const int sb = bc & 1;
            if (bc >= 2) {
              // the store that last used this buffer has finished reading it
              if (leader) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
              asm volatile("bar.sync 1, 128;" ::: "memory");
            }
            uint8_t* boxp = stg_base + (size_t)sb * (BM * 128) + row * 128;
#pragma unroll
            for (int h = 0; h < 2; h++) {
              const int c = bx * 32 + h * 16;
              if (c >= p.Rpad) break;
              float v[16], w[16];
              tmem_ld16(taddr + c, v);
              tmem_ld16(taddr + p.Rpad + c, w);           // lo-plane products
#pragma unroll
              for (int e = 0; e < 16; e++) v[e] += w[e];
#pragma unroll
              for (int g4 = 0; g4 < 4; g4++) {
                const int ch = h * 4 + g4;
                *reinterpret_cast<float4*>(boxp + ((ch ^ (row & 7)) << 4)) =
                    make_float4(v[4 * g4], v[4 * g4 + 1], v[4 * g4 + 2], v[4 * g4 + 3]);
              }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (leader) {
              tma_store_3d(&mapO, stg_u32 + sb * (BM * 128), bx * 32, (int)m0, zb);
              asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
          }
        } else {
          float* srow = stg + row * p.RS;
          for (int c = 0; c < p.Rpad; c += 16) {
            float v[16], w[16];
            tmem_ld16(taddr + c, v);
            tmem_ld16(taddr + p.Rpad + c, w);             // lo-plane products
#pragma unroll
            for (int e = 0; e < 16; e++) v[e] += w[e];
#pragma unroll
            for (int g4 = 0; g4 < 4; g4++)
              if (c + 4 * g4 < p.RS)
                *reinterpret_cast<float4*>(srow + c + 4 * g4) =
                    make_float4(v[4 * g4], v[4 * g4 + 1], v[4 * g4 + 2], v[4 * g4 + 3]);
          }
          asm volatile("bar.sync 1, 128;" ::: "memory");
          const int rows = (int)min((int64_t)BM, p.M - m0);
          float* gout = p.out + (((int64_t)z * p.batch + b) * p.M + m0) * p.R;
          for (int r2 = ew; r2 < rows; r2 += 4) {
            const float* sr = stg + r2 * p.RS;
            float* gr = gout + (int64_t)r2 * p.R;
            for (int col = lane; col < p.R; col += 32) gr[col] = sr[col];
          }
          asm volatile("bar.sync 1, 128;" ::: "memory");
        }
      }
      // every TMEM load of this unit has completed: the accumulators are free
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acce_bar[buf]));
    }
    if (p.tma_store && leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(tmem_cols)
                 : "memory");
  }
  // every CTA has taken its last unit: the last one out resets the counter
  if (threadIdx.x == 0 && p.sched) {
    __threadfence();
    if (atomicAdd(p.sched + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(p.sched, 0);
      atomicExch(p.sched + 1, 0);
    }
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
    else
      cudaGetLastError();
  });
  return fn;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

cudaError_t setup_umma_kernels() {
  const int smem = 227 * 1024 - 1024;
  cudaError_t e = cudaFuncSetAttribute(umma_gemm_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(umma_gemm_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

bool umma_supported(int64_t K, int64_t M, bool kmajor, int R) {
  if (R < 1 || R > 128) return false;
  if (K >= (1ll << 31) || M >= (1ll << 31)) return false;
  if (kmajor) return K % 8 == 0;
  return M % 8 == 0;
}

cudaError_t umma_gemm_bf16(const __nv_bfloat16* Xb, const __nv_bfloat16* Bt, float* out,
                           float* partials, int64_t batch, int64_t K, int64_t M, int R, int Rpad,
                           int64_t Kstride, bool kmajor, int splits, int* err_flag, int* sched,
                           Launch L, uint64_t wait_limit) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (!umma_supported(K, M, kmajor, R) || Rpad % 16 || Rpad > 128 || Rpad < R)
    return cudaErrorInvalidValue;
  if (kmajor && batch != 1) return cudaErrorInvalidValue;

  CUtensorMap mapA, mapB;
  CUresult cr;
  if (kmajor) {
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)M};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {BK, BM};
    cuuint32_t es[2] = {1, 1};
    cr = enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Xb, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t dims[3] = {(cuuint64_t)M, (cuuint64_t)K, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)M * 2, (cuuint64_t)M * K * 2};
    cuuint32_t box[3] = {64, BK, 1};
    cuuint32_t es[3] = {1, 1, 1};
    cr = enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)Xb, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  {
    // B: two planes (hi, lo) of Rpad rows x Kstride
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)Rpad, 2};
    cuuint64_t strides[2] = {(cuuint64_t)Kstride * 2, (cuuint64_t)Kstride * Rpad * 2};
    cuuint32_t box[3] = {BK, (cuuint32_t)Rpad, 2};
    cuuint32_t es[3] = {1, 1, 1};
    cr = enc(&mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)Bt, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;

  UmmaParams p;
  p.batch = batch;
  p.K = K;
  p.M = M;
  p.R = R;
  p.Rpad = Rpad;
  if (splits < 1) splits = 1;
  p.kchunk = cdiv(cdiv(K, splits), BK) * BK;
  p.splits = (int)cdiv(K, p.kchunk);
  p.mtiles = cdiv(M, BM);
  p.err = err_flag;
  p.sched = sched;
  p.wait_limit = wait_limit ? (unsigned long long)wait_limit : kTimeoutCycles;
  p.out = p.splits > 1 ? partials : out;
  int RS = (R + 3) / 4 * 4;
  if (((RS / 4) & 1) == 0) RS += 4;
  p.RS = RS;
  p.nbox = (Rpad + 31) / 32;
  p.tma_store = (R % 4 == 0) ? 1 : 0;
  const int staging = p.tma_store ? 2 * BM * 128 : BM * RS * 4;
  const int budget = 227 * 1024 - 2048;
  // two tiles per unit when there are two and three stages still fit
  auto stages_for = [&](int tpu) {
    return std::min(8, (budget - staging) / (tpu * A_STAGE_BYTES + 2 * Rpad * BK * 2));
  };
  // two tiles per unit (no double buffering then) only when every CTA gets
  // a single unit and three stages still fit
  p.tpu = (p.mtiles >= 2 && cdiv(p.mtiles, 2) * batch * p.splits <= num_sms() && stages_for(2) >= 3) ? 2 : 1;
  p.mgroups = cdiv(p.mtiles, p.tpu);
  p.units = p.mgroups * batch * p.splits;
  const int stage_bytes = p.tpu * A_STAGE_BYTES + 2 * Rpad * BK * 2;
  CUtensorMap mapO;
  memset(&mapO, 0, sizeof(mapO));
  if (p.tma_store) {
    // out viewed as [splits*batch][M][R] fp32; box 128 rows x 32 columns, swizzled
    cuuint64_t dims[3] = {(cuuint64_t)R, (cuuint64_t)M, (cuuint64_t)(batch * p.splits)};
    cuuint64_t strides[2] = {(cuuint64_t)R * 4, (cuuint64_t)M * R * 4};
    cuuint32_t box[3] = {32, BM, 1};
    cuuint32_t es[3] = {1, 1, 1};
    cr = enc(&mapO, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)p.out, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  p.stages = stages_for(p.tpu);
  if (p.stages < 2) return cudaErrorInvalidValue;
  const size_t smem = (size_t)p.stages * stage_bytes + staging + 1024;
  const int grid = (int)std::min<int64_t>(p.units, num_sms());

  cudaError_t e;
  if (kmajor)
    umma_gemm_kernel<true><<<grid, kThreadsUmma, smem, L.stream>>>(mapA, mapB, mapO, p);
  else
    umma_gemm_kernel<false><<<grid, kThreadsUmma, smem, L.stream>>>(mapA, mapB, mapO, p);
  (*L.counter)++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (p.splits > 1) {
    reduce_splits<float>(partials, out, batch * M * R, p.splits, L);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace cpals
