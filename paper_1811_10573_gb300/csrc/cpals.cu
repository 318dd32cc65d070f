// C ABI, context and the host-side plans of the dimension trees.
//
// Paper: Algorithm 1 (CP-ALS), Algorithm 3 (PP-CP-ALS), Sec. 2.5 (dimension
// tree for ALS), Sec. 3.2.3 (dimension tree for the PP operators), Eq. 3 (PP
// update), Sec. 5 (fitness).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cpals.h"
#include "ctrl_dev.cuh"
#include "internal.h"

using namespace cpals;

namespace {

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

enum GraphSlot { G_ALS = 0, G_PP_V = 1, G_PP_NOV = 2, G_BUILD = 3, G_FIT = 4, G_SLOTS = 5 };
constexpr int kEvPairs = 16;

}  // namespace

struct cpals_ctx {
  // problem
  int N = 0, R = 0, prec = 0;
  int dev = 0;          // device the context lives on
  int64_t dims[kMaxModes] = {0};
  int64_t total = 0;
  int h = 0;            // left half of the ALS tree: modes [0, h)
  // ALS variants (Sec. 5.1): update step size per mode (1 = plain ALS), and
  // ties tie[m2] = m1 < m2 (mode m2 shares mode m1's factor; -1 = none)
  double lam[kMaxModes] = {1, 1, 1, 1, 1, 1, 1, 1};
  int tie[kMaxModes] = {-1, -1, -1, -1, -1, -1, -1, -1};
  bool tied_any = false;
  int64_t PL = 1, PR = 1;
  int64_t smax = 0;
  int Rpad = 0;         // R rounded up to the tensor-core N granularity
  size_t esz = 0;       // bytes per compute-precision element

  // streams and errors
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;       // Cholesky factorisations overlap the contractions
  cudaStream_t user = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
  std::string err;

  // tensor
  void* X = nullptr;                 // float64 (FP64) or float32 (FP32, MIXED)
  __nv_bfloat16* Xb = nullptr;       // MIXED: bf16 copy
  double normX2 = 0.0;
  bool have_tensor = false, have_factors = false;

  // factors (float64 master copies) and compute-precision copies
  double* A[kMaxModes] = {nullptr};
  double* Ap[kMaxModes] = {nullptr};
  double* dA[kMaxModes] = {nullptr};
  void* Ac[kMaxModes] = {nullptr};
  void* dAc[kMaxModes] = {nullptr};
  bool dfm = false;      // FP32/mixed: double-float normal-equation kernels
  float* Alo[kMaxModes] = {nullptr};
  float* Aphi[kMaxModes] = {nullptr};
  float* Aplo[kMaxModes] = {nullptr};
  float* Shi = nullptr;  // N*R*R
  float* Slo = nullptr;
  float* Wf = nullptr;   // N*R*R (float W for the df path)
  float2* Linv = nullptr; // W = L^-1 of Gamma^(n), double-float, R x (R|1)
  float2* Gpk = nullptr;  // Gamma of the next mode, packed by columns (written by the Gram kernel)
  float* Zf = nullptr;   // R*R
  double* S = nullptr;   // N*R*R
  double* W = nullptr;   // N*R*R
  double* Lf = nullptr;  // R*R
  double* Z = nullptr;   // R*R

  // workspaces (compute precision unless noted)
  void* ML = nullptr;    // PL x R
  void* MR = nullptr;    // PR x R
  void* krp = nullptr;   // max(PL, PR) x R
  void* tmp[2] = {nullptr, nullptr};
  void* rhs = nullptr;   // smax x R
  void* rhs2 = nullptr;    // smax x R compute precision (allocated as float64)
  void* gpart = nullptr;   // split-K partials
  size_t gpart_bytes = 0;
  __nv_bfloat16* Bt = nullptr;   // MIXED: transposed bf16 B operand
  size_t Bt_elems = 0;
  double* rownorm = nullptr;     // 2*smax
  double* dscr[2] = {nullptr, nullptr};   // smax x R float64 scratch (inspection solves)
  double* dpart = nullptr;       // float64 partials (Grams, fitness, norms)
  double* scal = nullptr;        // device scalars
  double* scal_h = nullptr;      // pinned mirror
  int* status = nullptr;         // device status words
  int* tickets = nullptr;        // per-tile completion tickets of the Gram kernel
  int* status_h = nullptr;

  // PP operators
  bool pp_alloc = false, ops_built = false;
  void* ops[kMaxModes][kMaxModes] = {{nullptr}};
  void* Mp[kMaxModes] = {nullptr};
  std::vector<void*> lvl_bufs;                 // intermediate levels (freed with ctx)
  void* lvl[kMaxModes][kMaxModes][kMaxModes] = {{{nullptr}}};  // [l][i][j]

  // graphs, stats
  bool graphs = true;
  cudaGraphExec_t gexec[G_SLOTS] = {nullptr};
  int64_t gcount[G_SLOTS] = {0};
  int gev[G_SLOTS] = {0};
  bool profiling = false;
  cudaEvent_t ev0[kEvPairs] = {nullptr}, ev1[kEvPairs] = {nullptr};
  double ev_bytes[kEvPairs] = {0}, ev_flops[kEvPairs] = {0};
  int ev_kind[kEvPairs] = {0};     // 0: first-level contraction, 2: PP correction
  double gev_bytes[G_SLOTS][kEvPairs] = {{0}}, gev_flops[G_SLOTS][kEvPairs] = {{0}};
  int gev_kind[G_SLOTS][kEvPairs] = {{0}};
  int ev_used = 0;
  int64_t launches = 0;
  int64_t fl_launches = 0;
  double fl_ms = 0, fl_bytes = 0, fl_flops = 0;
  int64_t pc_launches = 0;         // PP correction launches timed with events
  double pc_ms = 0, pc_bytes = 0;
  int* umma_err = nullptr;
  uint64_t wait_limit = 0;         // bound of the tensor-core kernel's waits (cycles; 0 = default)
  int* umma_sched = nullptr;       // work counter of the tensor-core kernel (launches on stream)
  // learned controller
  float* ctrl_params = nullptr;    // device, ctrl_param_count(kCtrlFeatures) floats
  float* ctrl_io = nullptr;        // device: features (kCtrlFeatures) then probabilities
  float* ctrl_io_h = nullptr;      // pinned host mirror
  double ctrl_conf = 0.6;
  bool ctrl_on = false;
  // Algorithm 3 on device flags (cpals_run without a host round trip per
  // sweep): one graph per use_V value, a while loop around a switch over
  // the sweep kinds, its state and traces in device memory
  bool device_loop = true;
  double pp_stop_tol = 0.0;                // Algorithm 3's stopping test inside PP runs (0: off)
  double label_target = 0.0;               // controller log: label by the time to this fitness (0: off)
  bool ctrl_last_dev = false;              // the last controlled run took its decisions in the device loop
  int label_rollout = 0;                   // controller log: sweep cap of a trial to the target
  cudaGraphExec_t loop_exec[2] = {nullptr, nullptr};
  int64_t loop_count[2][4] = {{0}};        // kernels per branch (launch accounting)
  void* loop_state = nullptr;              // LoopState (device)
  void* loop_state_h = nullptr;            // pinned mirror
  double* loop_fit = nullptr;              // traces (device), loop_cap entries each
  double* loop_time = nullptr;
  int* loop_kind = nullptr;
  int loop_cap = 0;
  std::string loop_note;                   // why the device loop is unavailable ("" if it is)
  // snapshot of the sweep state (controller logs)
  std::vector<void*> snap_bufs;
  bool snap_ops = false;
  bool snap_built = false, snap_factors = false;

  Launch L() { return Launch{stream, &launches}; }
  Launch Lside() { return Launch{side, &launches}; }

  cpals_status fail(cpals_status st, const std::string& msg) {
    err = msg;
    return st;
  }
  cpals_status cuda_fail(const char* what, cudaError_t e) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return CPALS_E_CUDA;
  }
};

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return c->cuda_fail(#call, e_);    \
  } while (0)

#define CKS(expr)                                \
  do {                                           \
    cpals_status s_ = (expr);                    \
    if (s_ != CPALS_OK) return s_;               \
  } while (0)

namespace {

template <typename T>
T* P(void* p) {
  return static_cast<T*>(p);
}

cpals_status dalloc(cpals_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return c->fail(CPALS_E_OOM, std::string("cudaMalloc(") + std::to_string(bytes) +
                                    "): " + cudaGetErrorString(e));
  }
  return CPALS_OK;
}

// ---------------------------------------------------------------- stream join
struct Join {
  cpals_ctx* c;
  explicit Join(cpals_ctx* cc) : c(cc) {
    cudaEventRecord(c->ev_in, c->user);
    cudaStreamWaitEvent(c->stream, c->ev_in, 0);
  }
  ~Join() {
    cudaEventRecord(c->ev_out, c->stream);
    cudaStreamWaitEvent(c->user, c->ev_out, 0);
  }
};

// ---------------------------------------------------------------- profiling
void ev_begin(cpals_ctx* c, int idx) {
  if (c->profiling && idx < kEvPairs)
    cudaEventRecordWithFlags(c->ev0[idx], c->stream, cudaEventRecordExternal);
}
void ev_end(cpals_ctx* c, int idx, double bytes, double flops, int kind = 0) {
  if (c->profiling && idx < kEvPairs) {
    cudaEventRecordWithFlags(c->ev1[idx], c->stream, cudaEventRecordExternal);
    c->ev_bytes[idx] = bytes;
    c->ev_flops[idx] = flops;
    c->ev_kind[idx] = kind;
  }
}
// after the stream is synchronised: accumulate the recorded pairs
void ev_harvest(cpals_ctx* c) {
  if (!c->profiling) {
    c->ev_used = 0;
    return;
  }
  for (int i = 0; i < c->ev_used && i < kEvPairs; i++) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev0[i], c->ev1[i]) == cudaSuccess) {
      if (c->ev_kind[i] == 2) {
        c->pc_ms += ms;
        c->pc_launches++;
        c->pc_bytes += c->ev_bytes[i];
      } else {
        c->fl_ms += ms;
        c->fl_launches++;
        c->fl_bytes += c->ev_bytes[i];
        c->fl_flops += c->ev_flops[i];
      }
    } else {
      cudaGetLastError();
    }
  }
  c->ev_used = 0;
}

// ---------------------------------------------------------------- first-level contraction
// out = X contracted over the modes kmodes (contiguous block of modes) with
// their factors' Khatri-Rao product (Sec. 2.5; Sec. 3.2.3 level 2).
// kmajor: the contracted modes are the trailing ones (out is M x R, M = the rest);
// else out[b][m][r] with b = modes before, m = modes after the contracted block.
// tc_ok = false keeps a MIXED_BF16 contraction on the SIMT float32 kernels
// (float32 X).
template <typename T>
cpals_status contract_first(cpals_ctx* c, int k0, int nk, void* const* facs, T* out,
                            int64_t batch, int64_t K, int64_t M, bool kmajor, bool tc_ok = true) {
  const int R = c->R;
  const bool tc = c->prec == CPALS_MIXED_BF16 && tc_ok && umma_supported(K, M, kmajor, R);
  const size_t xsz = c->prec == CPALS_FP64 ? 8 : (tc ? 2 : 4);
  // algorithmic bytes: read X once, read B once, write the output once
  const double bytes = (double)batch * K * M * xsz + (double)batch * M * R * sizeof(T) +
                       (double)K * R * (tc ? 2 : sizeof(T));
  const double flops = 2.0 * batch * K * M * R;
  const int idx = c->ev_used++;
  // split K when the output alone does not fill the GPU
  const int64_t mtiles = cdiv(M, 128) * batch;
  int splits = 1;
  if (mtiles < 2 * 152) splits = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(2 * 152, mtiles), cdiv(K, 256)));
  while (splits > 1 && (size_t)splits * batch * M * R * sizeof(T) > c->gpart_bytes) splits--;
  if (!tc) {
    // float64 SIMT contractions are bound by the FP64 pipe: a grid of whole
    // waves of resident CTAs leaves no SM idle in a partial last wave
    const int ws = gemm_simt_wave_splits(batch, K, M, R, kmajor, sizeof(T),
                                         (int64_t)(c->gpart_bytes / sizeof(T)));
    if (ws > 0) splits = ws;
  }

  if (tc) {
    const float* fl[kMaxModes];
    for (int i = 0; i < nk; i++) fl[i] = P<const float>(facs[k0 + i]);
    const int64_t Kstride = cdiv(K, 8) * 8;
    khatri_rao_bf16_t(fl, c->dims + k0, nk, R, c->Rpad, Kstride, c->Bt, c->L());
    ev_begin(c, idx);
    CK(umma_gemm_bf16(c->Xb, c->Bt, P<float>(out), P<float>(c->gpart), batch, K, M, R, c->Rpad,
                      Kstride, kmajor, splits, c->umma_err, c->umma_sched, c->L(), c->wait_limit));
    ev_end(c, idx, bytes, flops);
    return CPALS_OK;
  }
  const T* B;
  if (nk == 1) {
    B = P<const T>(facs[k0]);
  } else {
    const T* fl[kMaxModes];
    for (int i = 0; i < nk; i++) fl[i] = P<const T>(facs[k0 + i]);
    khatri_rao<T>(fl, c->dims + k0, nk, R, P<T>(c->krp), c->L());
    B = P<const T>(c->krp);
  }
  ev_begin(c, idx);
  gemm_simt<T, T>(P<const T>(c->X), B, out, P<T>(c->gpart), batch, K, M, R, kmajor, splits, c->L(),
                  (int64_t)(c->gpart_bytes / sizeof(T)));
  ev_end(c, idx, bytes, flops);
  return CPALS_OK;
}

// Contract every mode of an intermediate except `keep` (multi-TTV chain,
// Sec. 2.5 lower levels).  in has modes `modes` (ascending) then r.
template <typename T>
const T* contract_chain(cpals_ctx* c, const T* in, std::vector<int> modes, int keep,
                        void* const* facs, T* final_out) {
  const T* cur = in;
  int ping = 0;
  while (modes.size() > 1) {
    int pos = (int)modes.size() - 1;
    if (modes[pos] == keep) pos--;
    const int w = modes[pos];
    int64_t outer = 1, inner = 1;
    for (int i = 0; i < pos; i++) outer *= c->dims[modes[i]];
    for (int i = pos + 1; i < (int)modes.size(); i++) inner *= c->dims[modes[i]];
    T* dst = modes.size() == 2 ? final_out : P<T>(c->tmp[ping]);
    ttv<T>(cur, P<const T>(facs[w]), dst, outer, (int)c->dims[w], inner, c->R, c->L());
    cur = dst;
    ping ^= 1;
    modes.erase(modes.begin() + pos);
  }
  return cur;
}

// Normal-equation update of mode n (Algorithm 1; the PP sweep of Algorithm 3
// when pp), in two halves: factor_async factors Gamma^(n) on the side
// stream (it needs only the Grams of the other modes), so it runs under the
// contraction that forms the right-hand side; finish_mode joins and solves.
void factor_async(cpals_ctx* c, int n, bool pp, bool useV) {
  cudaEventRecord(c->ev_fork, c->stream);
  cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  // with tied modes Gamma is formed from the Grams (the tied copies are in place)
  if (c->dfm)
    chol_df(c->Shi, c->Slo, c->Wf, c->tied_any ? nullptr : c->Gpk, c->N, n, c->R, c->Linv, c->Zf,
            pp && useV, c->status, c->Lside());
  else
    gamma_chol(c->S, c->W, c->N, n, c->R, c->Lf, c->Z, pp && useV, c->status, c->Lside());
  cudaEventRecord(c->ev_join, c->side);
}

template <typename T>
void finish_mode(cpals_ctx* c, int n, const T* rhs, bool pp, bool useV) {
  const int R = c->R;
  const int s = (int)c->dims[n];
  const bool v = pp && useV;
  const int64_t off = (int64_t)n * R * R;
  cudaStreamWaitEvent(c->stream, c->ev_join, 0);
  if (c->dfm) {
    float* Ahi = P<float>(c->Ac[n]);
    // the last mode's full M~ (with the second-order terms) for the PP
    // fitness estimate; the solve forms its own double-float sum
    if (v && n == c->N - 1) vterm_fz((const float*)rhs, Ahi, c->Zf, P<float>(c->rhs2), s, R, c->L());
    solve_df((const float*)rhs, c->A[n], Ahi, c->Alo[n], pp ? c->Aphi[n] : nullptr,
             pp ? c->Aplo[n] : nullptr, c->dA[n], P<float>(c->dAc[n]), c->Linv,
             v ? c->Zf : nullptr, (float2*)c->rownorm, s, R, n, c->lam[n], c->status, c->L());
    gram_df(Ahi, c->Alo[n], Ahi, P<const float>(c->dAc[n]), c->S + off, c->Shi + off,
            c->Slo + off, c->Wf + off, pp, s, R, (const float2*)c->rownorm, c->scal + 8 + 2 * n,
            c->Shi, c->Slo, c->N, n, c->tied_any ? -1 : (n + 1) % c->N, c->Gpk, c->L());
    return;
  }
  if (v)
    solve_rows_v<T>(rhs, c->A[n], c->Ap[n], c->dA[n], c->Lf, c->Z, P<T>(c->rhs2), P<T>(c->Ac[n]),
                    P<T>(c->dAc[n]), c->rownorm, s, R, n, c->lam[n], c->status, c->L());
  else
    solve_rows<T>(rhs, c->A[n], pp ? c->Ap[n] : nullptr, c->dA[n], c->Lf, P<T>(c->Ac[n]),
                  P<T>(c->dAc[n]), c->rownorm, s, R, n, c->lam[n], c->status, c->L());
  gram_update<T>(c->A[n], P<const T>(c->Ac[n]), P<const T>(c->dAc[n]), c->S + off, c->W + off,
                 pp, s, R, c->rownorm, c->scal + 8 + 2 * n, c->dpart, c->tickets, c->L());
}

// Symmetry constraint (Sec. 5.1, X = [[A, B, B]]): every mode tied to mode n
// takes mode n's new factor and its derived state (compute copies, change,
// Grams, W = A^T dA, norms) right after mode n's update; a tied mode is never
// solved for.
bool tied(const cpals_ctx* c, int n) { return c->tie[n] >= 0; }

cpals_status tie_copy(cpals_ctx* c, int n) {
  if (!c->tied_any) return CPALS_OK;
  const int R = c->R;
  auto cp = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream);
  };
  for (int m = 0; m < c->N; m++) {
    if (c->tie[m] != n) continue;
    const size_t sR = (size_t)c->dims[n] * R, RR = (size_t)R * R;
    const int64_t om = (int64_t)m * R * R, on = (int64_t)n * R * R;
    CK(cp(c->A[m], c->A[n], sR * 8));
    CK(cp(c->dA[m], c->dA[n], sR * 8));
    CK(cp(c->Ac[m], c->Ac[n], sR * c->esz));
    CK(cp(c->dAc[m], c->dAc[n], sR * c->esz));
    CK(cp(c->S + om, c->S + on, RR * 8));
    CK(cp(c->W + om, c->W + on, RR * 8));
    if (c->dfm) {
      CK(cp(c->Alo[m], c->Alo[n], sR * 4));
      CK(cp(c->Shi + om, c->Shi + on, RR * 4));
      CK(cp(c->Slo + om, c->Slo + on, RR * 4));
      CK(cp(c->Wf + om, c->Wf + on, RR * 4));
    }
    CK(cp(c->scal + 8 + 2 * m, c->scal + 8 + 2 * n, 2 * 8));
  }
  return CPALS_OK;
}

// ---------------------------------------------------------------- ALS sweep
template <typename T>
cpals_status als_sweep_launch(cpals_ctx* c) {
  const int N = c->N, h = c->h, R = c->R;
  std::vector<int> Lm, Rm;
  for (int k = 0; k < h; k++) Lm.push_back(k);
  for (int k = h; k < N; k++) Rm.push_back(k);
  // left half: M^(L) = X_(L) (A^(h) (.) ... (.) A^(N-1))
  // (mode 0 is never tied; a tied mode is skipped, except that the last
  // mode's right-hand side is still formed for the fitness)
  factor_async(c, 0, false, false);
  CKS(contract_first<T>(c, h, N - h, c->Ac, P<T>(c->ML), 1, c->PR, c->PL, true));
  for (int n = 0; n < h; n++) {
    if (tied(c, n)) continue;
    if (n > 0) factor_async(c, n, false, false);
    const T* rhs = contract_chain<T>(c, P<const T>(c->ML), Lm, n, c->Ac, P<T>(c->rhs));
    finish_mode<T>(c, n, rhs, false, false);
    CKS(tie_copy(c, n));
  }
  // right half with the updated left factors: M^(Rt) = X_(L)^T (A^(0) (.) ... (.) A^(h-1))
  if (!tied(c, h)) factor_async(c, h, false, false);
  CKS(contract_first<T>(c, 0, h, c->Ac, P<T>(c->MR), 1, c->PL, c->PR, false));
  const T* last = nullptr;
  for (int n = h; n < N; n++) {
    if (tied(c, n)) {
      if (n == N - 1) last = contract_chain<T>(c, P<const T>(c->MR), Rm, n, c->Ac, P<T>(c->rhs));
      continue;
    }
    if (n > h) factor_async(c, n, false, false);
    last = contract_chain<T>(c, P<const T>(c->MR), Rm, n, c->Ac, P<T>(c->rhs));
    finish_mode<T>(c, n, last, false, false);
    CKS(tie_copy(c, n));
  }
  fitness<T>(last, c->A[N - 1], c->S, N, R, (int)c->dims[N - 1], c->scal + 40, c->scal, c->dpart,
             c->tickets + 62, c->L());
  return CPALS_OK;
}

// exact M^(n) at the current factors into a buffer; returns the pointer
template <typename T>
cpals_status mttkrp_launch(cpals_ctx* c, int n, const T** result) {
  const int N = c->N, h = c->h;
  std::vector<int> modes;
  if (n < h) {
    for (int k = 0; k < h; k++) modes.push_back(k);
    CKS(contract_first<T>(c, h, N - h, c->Ac, P<T>(c->ML), 1, c->PR, c->PL, true));
    *result = contract_chain<T>(c, P<const T>(c->ML), modes, n, c->Ac, P<T>(c->rhs));
  } else {
    for (int k = h; k < N; k++) modes.push_back(k);
    CKS(contract_first<T>(c, 0, h, c->Ac, P<T>(c->MR), 1, c->PL, c->PR, false));
    *result = contract_chain<T>(c, P<const T>(c->MR), modes, n, c->Ac, P<T>(c->rhs));
  }
  return CPALS_OK;
}

template <typename T>
cpals_status fitness_launch(cpals_ctx* c) {
  const T* last = nullptr;
  CKS(mttkrp_launch<T>(c, c->N - 1, &last));
  fitness<T>(last, c->A[c->N - 1], c->S, c->N, c->R, (int)c->dims[c->N - 1], c->scal + 40, c->scal,
             c->dpart, c->tickets + 62, c->L());
  return CPALS_OK;
}

// ---------------------------------------------------------------- PP operators
// Level-l tensors hold modes {i, j} U {l+1, ..., N-1} (0-based), i < j <= l
// (Sec. 3.2.3).  Level 1 is X itself.
std::vector<int> level_modes(int N, int l, int i, int j) {
  std::vector<int> m = {i, j};
  for (int k = l + 1; k < N; k++) m.push_back(k);
  return m;
}

// parent of (i,j) at level l (a tensor at level l-1) and the mode contracted
void tree_parent(int l, int i, int j, int* pi, int* pj, int* w) {
  if (j <= l - 1) {
    *pi = i; *pj = j; *w = l;
  } else if (i < l - 1) {
    *pi = i; *pj = l - 1; *w = l - 1;
  } else {
    *pi = l - 2; *pj = l - 1; *w = l - 2;
  }
}

template <typename T>
cpals_status pp_alloc(cpals_ctx* c) {
  if (c->pp_alloc) return CPALS_OK;
  const int N = c->N, R = c->R;
  for (int i = 0; i < N; i++)
    for (int n = i + 1; n < N; n++)
      CKS(dalloc(c, &c->ops[i][n], (size_t)c->dims[i] * c->dims[n] * R * sizeof(T)));
  for (int n = 0; n < N; n++) CKS(dalloc(c, &c->Mp[n], (size_t)c->dims[n] * R * sizeof(T)));
  for (int l = 2; l <= N - 2; l++)
    for (int i = 0; i <= l; i++)
      for (int j = i + 1; j <= l; j++) {
        int64_t sz = R;
        for (int m : level_modes(N, l, i, j)) sz *= c->dims[m];
        void* p = nullptr;
        CKS(dalloc(c, &p, (size_t)sz * sizeof(T)));
        c->lvl_bufs.push_back(p);
        c->lvl[l][i][j] = p;
      }
  c->pp_alloc = true;
  return CPALS_OK;
}

template <typename T>
cpals_status pp_build_launch(cpals_ctx* c) {
  const int N = c->N, R = c->R;
  // level 2: three first-level contractions of X (modes 2, 1, 0)
  for (int w = 2; w >= 0; w--) {
    int i, j;
    if (w == 2) { i = 0; j = 1; } else if (w == 1) { i = 0; j = 2; } else { i = 1; j = 2; }
    T* dst = P<T>(N == 3 ? c->ops[i][j] : c->lvl[2][i][j]);
    int64_t batch = 1, M = 1;
    for (int k = 0; k < w; k++) batch *= c->dims[k];
    for (int k = w + 1; k < N; k++) M *= c->dims[k];
    const bool kmajor = (w == N - 1);
    if (kmajor) { M = batch; batch = 1; }
    // a short contracted mode (K below 64) with a large output leaves the
    // tcgen05 kernel nothing but its per-tile cost (the TMEM round trip and
    // epilogue of every 128-row tile): measured 2.76 ms per launch against
    // 1.05 ms on the SIMT float32 kernel for the 24^6 tree's K = 24 (the
    // operators then carry float32 X in MIXED_BF16)
    CKS(contract_first<T>(c, w, 1, c->Ac, dst, batch, c->dims[w], M, kmajor, c->dims[w] >= 64));
  }
  // levels 3 .. N-1: one multi-TTV per child
  for (int l = 3; l <= N - 1; l++) {
    for (int i = 0; i <= l; i++)
      for (int j = i + 1; j <= l; j++) {
        int pi, pj, w;
        tree_parent(l, i, j, &pi, &pj, &w);
        const std::vector<int> pm = level_modes(N, l - 1, pi, pj);
        int pos = 0;
        while (pm[pos] != w) pos++;
        int64_t outer = 1, inner = 1;
        for (int k = 0; k < pos; k++) outer *= c->dims[pm[k]];
        for (int k = pos + 1; k < (int)pm.size(); k++) inner *= c->dims[pm[k]];
        const T* src = P<const T>(c->lvl[l - 1][pi][pj]);
        T* dst = P<T>(l == N - 1 ? c->ops[i][j] : c->lvl[l][i][j]);
        ttv<T>(src, P<const T>(c->Ac[w]), dst, outer, (int)c->dims[w], inner, R, c->L());
      }
  }
  // M_p^(n) from a leaf (Sec. 3.2.3: contract M_p^(i,n) with A_p^(i))
  for (int n = 0; n < N; n++) {
    if (n == 0)
      ttv<T>(P<const T>(c->ops[0][1]), P<const T>(c->Ac[1]), P<T>(c->Mp[0]), c->dims[0],
             (int)c->dims[1], 1, R, c->L());
    else
      ttv<T>(P<const T>(c->ops[0][n]), P<const T>(c->Ac[0]), P<T>(c->Mp[n]), 1, (int)c->dims[0],
             c->dims[n], R, c->L());
  }
  // A_p <- A, dA <- 0 (the PP initialisation of Algorithm 3)
  for (int n = 0; n < N; n++) {
    const size_t sR = (size_t)c->dims[n] * R;
    CK(cudaMemcpyAsync(c->Ap[n], c->A[n], sR * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(c->dA[n], 0, sR * sizeof(double), c->stream));
    CK(cudaMemsetAsync(c->dAc[n], 0, sR * c->esz, c->stream));
  }
  CK(cudaMemsetAsync(c->W, 0, (size_t)N * R * R * sizeof(double), c->stream));
  if (c->dfm) {
    CK(cudaMemsetAsync(c->Wf, 0, (size_t)N * R * R * sizeof(float), c->stream));
    for (int n = 0; n < N; n++) {
      const size_t sR = (size_t)c->dims[n] * R;
      CK(cudaMemcpyAsync(c->Aphi[n], c->Ac[n], sR * 4, cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(c->Aplo[n], c->Alo[n], sR * 4, cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  // ||dA^(n)||^2 <- 0; ||A^(n)||^2 is unchanged
  for (int n = 0; n < N; n++)
    CK(cudaMemsetAsync(c->scal + 8 + 2 * n, 0, sizeof(double), c->stream));
  return CPALS_OK;
}

// ---------------------------------------------------------------- PP sweep
template <typename T>
void pp_terms(cpals_ctx* c, int n, PPTerm<T>* terms) {
  const int N = c->N, R = c->R;
  int t = 0;
  for (int i = 0; i < N; i++) {
    if (i == n) continue;
    PPTerm<T> tt;
    tt.dA = P<const T>(c->dAc[i]);
    tt.sx = (int)c->dims[i];
    if (i < n) {        // M_p^(i,n)(x, y, r)
      tt.op = P<const T>(c->ops[i][n]);
      tt.xstride = c->dims[n] * R;
      tt.ystride = R;
    } else {            // M_p^(n,i)(y, x, r)
      tt.op = P<const T>(c->ops[n][i]);
      tt.xstride = R;
      tt.ystride = c->dims[i] * R;
    }
    terms[t++] = tt;
  }
}

template <typename T>
cpals_status pp_sweep_launch(cpals_ctx* c, bool useV) {
  const int N = c->N, R = c->R;
  PPTerm<T> terms[kMaxModes];
  for (int n = 0; n < N; n++) {
    const bool skip = tied(c, n);
    if (skip && n != N - 1) continue;
    if (!skip) factor_async(c, n, true, useV);
    pp_terms<T>(c, n, terms);
    // algorithmic bytes: every operator and dA^(i) once, M_p^(n) once, the result once
    double pcb = 2.0 * (double)c->dims[n] * R * sizeof(T);
    for (int i = 0; i < N; i++)
      if (i != n) pcb += ((double)c->dims[i] * c->dims[n] * R + (double)c->dims[i] * R) * sizeof(T);
    const int idx = c->ev_used++;
    ev_begin(c, idx);
    pp_correct<T>(P<const T>(c->Mp[n]), terms, N - 1, P<T>(c->rhs), (int)c->dims[n], R, c->L());
    ev_end(c, idx, pcb, 0.0, 2);
    if (skip) continue;                 // a tied last mode: M~ only feeds the fitness estimate
    finish_mode<T>(c, n, P<const T>(c->rhs), true, useV);
    CKS(tie_copy(c, n));
  }
  // fitness estimate from M~^(N) (the last mode's right-hand side with the
  // second-order terms when they are on; the updated factors); a tied last
  // mode, which is not solved for, has only the first-order part
  const bool full = useV && !tied(c, N - 1);
  fitness<T>(P<const T>(full ? c->rhs2 : c->rhs), c->A[N - 1], c->S, N, R, (int)c->dims[N - 1], c->scal + 40,
             c->scal, c->dpart, c->tickets + 62, c->L());
  return CPALS_OK;
}

// ---------------------------------------------------------------- dispatch helpers
template <typename F>
cpals_status run_slot(cpals_ctx* c, int slot, F&& body) {
  if (!c->graphs) {
    c->ev_used = 0;
    return body();
  }
  if (!c->gexec[slot]) {
    cudaGraph_t g = nullptr;
    const int64_t before = c->launches;
    c->ev_used = 0;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cpals_status st = body();
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != CPALS_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return c->cuda_fail("cudaStreamEndCapture", e);
    e = cudaGraphInstantiate(&c->gexec[slot], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->gexec[slot] = nullptr;
      return c->cuda_fail("cudaGraphInstantiate", e);
    }
    c->gcount[slot] = c->launches - before;
    c->gev[slot] = c->ev_used;
    for (int i = 0; i < kEvPairs; i++) {
      c->gev_bytes[slot][i] = c->ev_bytes[i];
      c->gev_flops[slot][i] = c->ev_flops[i];
      c->gev_kind[slot][i] = c->ev_kind[i];
    }
    c->launches = before;
  }
  CK(cudaGraphLaunch(c->gexec[slot], c->stream));
  c->launches += c->gcount[slot];
  c->ev_used = c->gev[slot];
  for (int i = 0; i < kEvPairs; i++) {
    c->ev_bytes[i] = c->gev_bytes[slot][i];
    c->ev_flops[i] = c->gev_flops[slot][i];
    c->ev_kind[i] = c->gev_kind[slot][i];
  }
  return CPALS_OK;
}

void drop_graphs(cpals_ctx* c) {
  for (int i = 0; i < G_SLOTS; i++)
    if (c->gexec[i]) {
      cudaGraphExecDestroy(c->gexec[i]);
      c->gexec[i] = nullptr;
    }
  for (int i = 0; i < 2; i++)
    if (c->loop_exec[i]) {
      cudaGraphExecDestroy(c->loop_exec[i]);
      c->loop_exec[i] = nullptr;
    }
}

cpals_status sync_read(cpals_ctx* c) {
  CK(cudaMemcpyAsync(c->scal_h, c->scal, sizeof(double) * 32, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->status_h, c->status, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  ev_harvest(c);
  if (c->status_h[1])
    return c->fail(CPALS_E_TIMEOUT, "tensor-core contraction: a bounded wait gave up (code " +
                                        std::to_string(c->status_h[1]) + ")");
  if (c->status_h[2])
    return c->fail(CPALS_E_TIMEOUT, "row solve: the bulk copy of the factor did not complete");
  return CPALS_OK;
}

cpals_status check_status(cpals_ctx* c) {
  // a non-finite value (e.g. from a NaN or Inf in the input) is reported
  // before a failed factorisation it may have caused
  for (int n = 0; n < c->N; n++)
    if (!std::isfinite(c->scal_h[8 + 2 * n]) || !std::isfinite(c->scal_h[9 + 2 * n]))
      return c->fail(CPALS_E_NUMERIC, "non-finite factor in mode " + std::to_string(n));
  if (!std::isfinite(c->scal_h[0]))
    return c->fail(CPALS_E_NUMERIC, "non-finite fitness");
  if (c->status_h[0] & 0xffff) {        // bits 16 + n: Gamma^dagger used (not an error)
    const int bits = c->status_h[0] & 0xffff;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int) * 4, c->stream));
    return c->fail(CPALS_E_SINGULAR, "Gamma not finite for mode mask " + std::to_string(bits) +
                                         "; those factors were left unchanged");
  }
  return CPALS_OK;
}

bool is64(const cpals_ctx* c) { return c->prec == CPALS_FP64; }

cpals_status ready(cpals_ctx* c) {
  if (!c) return CPALS_E_INVALID;
  if (!c->have_tensor) return c->fail(CPALS_E_STATE, "no tensor: call cpals_set_tensor first");
  if (!c->have_factors) return c->fail(CPALS_E_STATE, "no factors: call cpals_init_factors first");
  return CPALS_OK;
}

template <typename T>
cpals_status copy_out(cpals_ctx* c, const T* src, int64_t n, double* out) {
  if (sizeof(T) == 8) {
    CK(cudaMemcpyAsync(out, src, n * 8, cudaMemcpyDeviceToHost, c->stream));
  } else {
    std::vector<float> tmp(n);
    CK(cudaMemcpyAsync(tmp.data(), src, n * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int64_t i = 0; i < n; i++) out[i] = tmp[i];
  }
  CK(cudaStreamSynchronize(c->stream));
  return CPALS_OK;
}

cpals_status do_als(cpals_ctx* c) {
  return run_slot(c, G_ALS, [&]() { return is64(c) ? als_sweep_launch<double>(c) : als_sweep_launch<float>(c); });
}
cpals_status do_build(cpals_ctx* c) {
  CKS(is64(c) ? pp_alloc<double>(c) : pp_alloc<float>(c));
  return run_slot(c, G_BUILD, [&]() { return is64(c) ? pp_build_launch<double>(c) : pp_build_launch<float>(c); });
}
cpals_status do_pp(cpals_ctx* c, bool useV) {
  return run_slot(c, useV ? G_PP_V : G_PP_NOV,
                  [&]() { return is64(c) ? pp_sweep_launch<double>(c, useV) : pp_sweep_launch<float>(c, useV); });
}
cpals_status do_fit(cpals_ctx* c) {
  return run_slot(c, G_FIT, [&]() { return is64(c) ? fitness_launch<double>(c) : fitness_launch<float>(c); });
}

bool all_small(const cpals_ctx* c, double eps) {
  for (int n = 0; n < c->N; n++) {
    const double d = std::sqrt(c->scal_h[8 + 2 * n]), a = std::sqrt(c->scal_h[9 + 2 * n]);
    if (!(d < eps * a)) return false;
  }
  return true;
}

// ---------------------------------------------------------------- snapshot
// The state a sweep reads and writes: factors (float64 masters, compute and
// double-float copies), A_p, dA, Grams, W, the next mode's packed Gamma and
// the device scalars; with ops also the PP operators and M_p (a rebuild
// overwrites them).  Buffers are allocated on first use and kept.
struct Region {
  void* p;
  size_t bytes;
};
std::vector<Region> state_regions(cpals_ctx* c, bool ops) {
  std::vector<Region> r;
  const int N = c->N, R = c->R;
  for (int n = 0; n < N; n++) {
    const size_t sR = (size_t)c->dims[n] * R;
    r.push_back({c->A[n], sR * 8});
    r.push_back({c->Ap[n], sR * 8});
    r.push_back({c->dA[n], sR * 8});
    r.push_back({c->Ac[n], sR * c->esz});
    r.push_back({c->dAc[n], sR * c->esz});
    if (c->dfm || c->Alo[n]) {
      if (c->Alo[n]) r.push_back({c->Alo[n], sR * 4});
      if (c->Aphi[n]) r.push_back({c->Aphi[n], sR * 4});
      if (c->Aplo[n]) r.push_back({c->Aplo[n], sR * 4});
    }
  }
  r.push_back({c->S, (size_t)N * R * R * 8});
  r.push_back({c->W, (size_t)N * R * R * 8});
  if (c->Shi) r.push_back({c->Shi, (size_t)N * R * R * 4});
  if (c->Slo) r.push_back({c->Slo, (size_t)N * R * R * 4});
  if (c->Wf) r.push_back({c->Wf, (size_t)N * R * R * 4});
  if (c->Gpk) r.push_back({c->Gpk, (size_t)R * (R + 1) / 2 * 8});
  r.push_back({c->scal, 32 * 8});
  if (ops && c->pp_alloc) {
    for (int i = 0; i < N; i++)
      for (int n = i + 1; n < N; n++) r.push_back({c->ops[i][n], (size_t)c->dims[i] * c->dims[n] * R * c->esz});
    for (int n = 0; n < N; n++) r.push_back({c->Mp[n], (size_t)c->dims[n] * R * c->esz});
  }
  return r;
}

cpals_status snapshot_take(cpals_ctx* c, bool ops) {
  const std::vector<Region> reg = state_regions(c, ops);
  while (c->snap_bufs.size() < reg.size()) c->snap_bufs.push_back(nullptr);
  for (size_t i = 0; i < reg.size(); i++) {
    if (!c->snap_bufs[i]) CKS(dalloc(c, &c->snap_bufs[i], reg[i].bytes));
    CK(cudaMemcpyAsync(c->snap_bufs[i], reg[i].p, reg[i].bytes, cudaMemcpyDeviceToDevice, c->stream));
  }
  c->snap_ops = ops && c->pp_alloc;
  c->snap_built = c->ops_built;
  c->snap_factors = c->have_factors;
  return CPALS_OK;
}

cpals_status snapshot_restore(cpals_ctx* c) {
  const std::vector<Region> reg = state_regions(c, c->snap_ops);
  for (size_t i = 0; i < reg.size() && i < c->snap_bufs.size(); i++)
    CK(cudaMemcpyAsync(reg[i].p, c->snap_bufs[i], reg[i].bytes, cudaMemcpyDeviceToDevice, c->stream));
  c->ops_built = c->snap_built;
  c->have_factors = c->snap_factors;
  return CPALS_OK;
}

// ---------------------------------------------------------------- controller features
constexpr int kCtrlHorizon = 4;   // sweeps per trial in the controller log

struct CtrlHist {
  double maxlr[2] = {0, 0};        // largest log10 dA ratio of the last two sweeps
  double res[4] = {-1, -1, -1, -1}; // residual 1 - f of the last four sweeps (newest first; -1: none)
  int since_build = 0;
  bool pp_ready = false;           // operators built and only PP sweeps since
  int last = -1;
  void push(cpals_ctx* c, int action, double fitness) {
    double m = -12;
    for (int n = 0; n < c->N; n++) {
      const double d = std::sqrt(c->scal_h[8 + 2 * n]), a = std::sqrt(c->scal_h[9 + 2 * n]);
      m = std::max(m, std::log10(std::max(d / std::max(a, 1e-300), 1e-12)));
    }
    maxlr[1] = maxlr[0];
    maxlr[0] = m;
    for (int k = 3; k > 0; k--) res[k] = res[k - 1];
    res[0] = 1.0 - fitness;
    last = action;
    if (action == ACT_ALS) {
      pp_ready = false;
      since_build = 0;
    } else if (action == ACT_REBUILD) {
      pp_ready = true;
      since_build = 1;
    } else {
      since_build++;
    }
  }
};

// The controller's input (kCtrlFeatures values, all O(1)): the per-mode log10
// ||dA||/||A|| (padded to 8 modes), the largest one of the two previous
// sweeps, log10 of the last three residual decreases, sweeps since the
// operators were built, whether a PP sweep is possible, the last action
// (one-hot), log10 eps and log10 of the current residual.
void ctrl_features(cpals_ctx* c, const CtrlHist& h, double eps, float* x) {
  for (int i = 0; i < kCtrlFeatures; i++) x[i] = 0.f;
  for (int n = 0; n < c->N && n < 8; n++) {
    const double d = std::sqrt(c->scal_h[8 + 2 * n]), a = std::sqrt(c->scal_h[9 + 2 * n]);
    const double lr = std::log10(std::max(d / std::max(a, 1e-300), 1e-12));
    x[n] = (float)(std::min(std::max(lr, -12.0), 2.0) / 4.0);
  }
  x[8] = (float)(h.maxlr[0] / 4.0);
  x[9] = (float)(h.maxlr[1] / 4.0);
  for (int k = 0; k < 3; k++) {
    const bool have = h.res[k] >= 0 && h.res[k + 1] >= 0;
    const double dec = have ? std::max(h.res[k + 1] - h.res[k], 1e-16) : 1e-16;
    x[10 + k] = (float)(std::log10(dec) / 8.0);
  }
  x[13] = (float)(h.pp_ready ? std::min(h.since_build, 20) / 10.0 : 0.0);
  x[14] = h.pp_ready ? 1.f : 0.f;
  if (h.last >= 0) x[15 + h.last] = 1.f;
  x[18] = (float)(std::log10(std::max(eps, 1e-12)) / 2.0);
  x[19] = (float)(std::log10(std::max(h.res[0] >= 0 ? h.res[0] : 1.0, 1e-16)) / 8.0);
}

// one sweep of the given kind; leaves the scalars read back
cpals_status do_action(cpals_ctx* c, int a, bool useV) {
  if (a == ACT_REBUILD) {
    CKS(do_build(c));
    c->ops_built = true;
    CKS(do_pp(c, useV));
  } else if (a == ACT_PP) {
    CKS(do_pp(c, useV));
  } else {
    CKS(do_als(c));
  }
  CKS(sync_read(c));
  return check_status(c);
}

// exact fitness of the current factors (Sec. 5)
cpals_status exact_fitness(cpals_ctx* c, double* f) {
  CKS(do_fit(c));
  CKS(sync_read(c));
  *f = c->scal_h[0];
  return CPALS_OK;
}

// ---------------------------------------------------------------- Algorithm 3 on the device
// The eps test of Algorithm 3 and the target test taken on the GPU: one CUDA
// graph per run holds a while loop (handle hw) whose body selects the next
// step with a switch (handle hs) over four captured bodies -- 0: ALS sweep,
// 1: operator build + PP sweep (the PP initialisation sweep), 2: PP sweep,
// 3: exact fitness (confirms a PP estimate that reached the target) -- and
// then decides the following step from the device scalars.  The decisions
// are those of the host loop of cpals_run: after an ALS sweep the operators
// are built iff every ||dA^(n)|| < eps ||A^(n)||; after a PP sweep another PP
// sweep follows iff that still holds, else one ALS sweep.  The loop ends at
// the sweep budget, at a confirmed target or at an error.
struct LoopState {
  int t;            // sweeps done
  int next;         // branch of the next iteration
  int hit;          // target confirmed
  int err;          // 0; 1 non-finite value; 2 Gamma not positive definite; 3 a bounded wait gave up
  int pending;      // kind of the PP sweep whose estimate awaits the exact fitness
  int confirms;     // exact-fitness branches run
  int max_sweeps;
  int N;
  double eps, target, pending_f;
  double tol;       // PP runs end when a sweep gains less fitness than this (0: off)
  double f_last, f_prev;   // fitness the algorithm saw after the last two sweeps
  int in_run;       // PP sweeps of the current PP run up to the last sweep (0 after ALS)
  unsigned long long t0;
  // learned controller (cpals_run_controlled): on/off, confidence,
  // parameters, its history, whether it took the next decision
  int ctrl;
  int src_next;
  double conf;
  const float* params;
  CtrlState ch;
  float last_x[20], last_p[3];   // the controller's last input and output
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool loop_all_small(const LoopState* s, const double* scal) {
  if (!(s->eps > 0.0)) return false;
  for (int n = 0; n < s->N; n++)
    if (!(sqrt(scal[8 + 2 * n]) < s->eps * sqrt(scal[9 + 2 * n]))) return false;
  return true;
}

// The learned controller's decision (as cpals_run_controlled's host loop):
// the network's most probable action when its probability reaches the
// confidence and it is not a PP sweep without valid operators, else the
// rule's branch; returns the branch (0 ALS, 1 rebuild + PP, 2 PP) on every
// lane.  One warp: lane i forms feature i from the history and the modes'
// lr (ctrl_mode_lr, shared), lane j hidden unit j.
__device__ int loop_ctrl_choose(LoopState* s, const double* lr, int rule_branch) {
  __shared__ float x[20], hsm[32], pr[3];
  __shared__ int out;
  const int lane = threadIdx.x & 31;
  if (lane < 20) {
    // the history as a local copy (features formed through the loop state's
    // pointer came out as those of the run's first decision in this kernel)
    const CtrlState h = s->ch;
    x[lane] = ctrl_feature(h, lr, s->N, s->eps, lane);
  }
  __syncwarp();
  mlp_probs_warp<20>(s->params, x, hsm, pr);
  if (lane == 0) {
    for (int i = 0; i < 20; i++) s->last_x[i] = x[i];
    for (int i = 0; i < 3; i++) s->last_p[i] = pr[i];
    int best = 0;
    for (int k = 1; k < 3; k++)
      if (pr[k] > pr[best]) best = k;
    s->src_next = 0;
    out = rule_branch;
    if (pr[best] >= s->conf && !(best == ACT_PP && !s->ch.pp_ready)) {
      s->src_next = 1;
      out = best == ACT_ALS ? 0 : (best == ACT_REBUILD ? 1 : 2);
    }
  }
  __syncwarp();
  return out;
}

// lr[n] = ctrl_mode_lr of the current scalars, mode n on lane n (the whole
// warp calls it; shared lr visible on return)
__device__ void loop_mode_lr(const LoopState* s, const double* scal, double* lr) {
  const int lane = threadIdx.x & 31, N = s->N;
  if (lane < N) lr[lane] = ctrl_mode_lr(scal, lane);
  __syncwarp();
}

// One warp (the node's 32 threads): lane 0 runs the rule, the warp the
// controller when there is one.
__global__ void loop_init_kernel(LoopState* s, const double* scal, cudaGraphConditionalHandle hw,
                                 cudaGraphConditionalHandle hs) {
  if (threadIdx.x >= 32 || blockIdx.x != 0) return;
  __shared__ int ask, rule;
  __shared__ double lr[kMaxModes];
  if (s->ctrl) loop_mode_lr(s, scal, lr);
  if (threadIdx.x == 0) {
    s->t = 0;
    s->hit = 0;
    s->err = 0;
    s->confirms = 0;
    s->f_last = s->f_prev = -1e300;
    s->in_run = 0;
    s->next = loop_all_small(s, scal) ? 1 : 0;   // the test at the head of the first sweep
    s->src_next = 0;
    if (s->ctrl) ctrl_state_start(s->ch, scal[0]);
    ask = s->ctrl;
    rule = s->next;
  }
  __syncwarp();
  if (ask) {
    const int nx = loop_ctrl_choose(s, lr, rule);
    if (threadIdx.x == 0) s->next = nx;
  }
  if (threadIdx.x == 0) {
    s->t0 = global_ns();
    cudaGraphSetConditional(hs, (unsigned)s->next);
    cudaGraphSetConditional(hw, s->max_sweeps > 0 ? 1u : 0u);
  }
}

// Lane 0's part of the decision after a sweep: records the sweep, ends the
// loop or sets the rule's next branch.  Returns 1 when the learned
// controller is to take the decision (the caller sets the switch then).
__device__ int loop_decide_rule(LoopState* s, const double* scal, const double* lr, const int* status,
                                double* ftr, int* ktr, double* ttr, cudaGraphConditionalHandle hw,
                                cudaGraphConditionalHandle hs) {
  int ran = s->next;
  const double f = scal[0];
  auto record = [&](int kind, double fv) {
    const int t = s->t;
    ftr[t] = fv;
    ktr[t] = kind | (s->src_next << 4);        // bit 4: the learned controller chose this sweep
    ttr[t] = (double)(global_ns() - s->t0) * 1e-9;
    s->t = t + 1;
    s->f_prev = s->f_last;
    s->f_last = fv;
    s->in_run = kind == 0 ? 0 : (kind == 1 ? 1 : s->in_run + 1);
    if (s->ctrl) ctrl_push(s->ch, lr, s->N, kind == 0 ? ACT_ALS : (kind == 1 ? ACT_REBUILD : ACT_PP), fv);
  };
  bool stop = false;
  if (ran == 3) {
    // the exact fitness of the factors a PP sweep left
    s->confirms++;
    if (f >= s->target) {
      s->hit = 1;
      record(s->pending, f);
    } else {
      record(s->pending, s->pending_f);
    }
    ran = s->pending;
  } else {
    if (status[1] || status[2]) {
      s->err = 3;                   // not recorded, as the host loop does
      stop = true;
    } else {
      bool finite = isfinite(f);
      for (int n = 0; n < s->N; n++)
        finite = finite && isfinite(scal[8 + 2 * n]) && isfinite(scal[9 + 2 * n]);
      if (!finite || (status[0] & 0xffff)) {
        s->err = finite ? 2 : 1;
        record(ran, f);
        stop = true;
      } else if (ran != 0 && s->target > 0.0 && f >= s->target) {
        // a PP estimate at the target: confirm with the exact fitness first
        s->pending = ran;
        s->pending_f = f;
        s->next = 3;
        cudaGraphSetConditional(hs, 3u);
        cudaGraphSetConditional(hw, 1u);
        return 0;
      } else {
        if (ran == 0 && s->target > 0.0 && f >= s->target) s->hit = 1;
        record(ran, f);
      }
    }
  }
  if (stop || s->hit || s->t >= s->max_sweeps) {
    cudaGraphSetConditional(hw, 0u);
    return 0;
  }
  const bool small = loop_all_small(s, scal);
  // from the third sweep of a PP run on, the stopping test also asks the
  // last PP sweep for a gain of tol over the one before it
  const bool gain = !(s->tol > 0.0) || s->in_run < 2 || s->f_last - s->f_prev >= s->tol;
  s->next = ran != 0 ? ((small && gain) ? 2 : 0) : (small ? 1 : 0);
  if (s->ctrl) return 1;
  cudaGraphSetConditional(hs, (unsigned)s->next);
  cudaGraphSetConditional(hw, 1u);
  return 0;
}

// The switch's value persists between iterations (its handle has no default
// assignment): each decision sets it for the next iteration.
__global__ void loop_decide_kernel(LoopState* s, const double* scal, const int* status, double* ftr,
                                   int* ktr, double* ttr, cudaGraphConditionalHandle hw,
                                   cudaGraphConditionalHandle hs) {
  if (threadIdx.x >= 32 || blockIdx.x != 0) return;
  __shared__ int ask, rule;
  __shared__ double lr[kMaxModes];
  // the modes' lr of the sweep just done: its record and the next features
  if (s->ctrl) loop_mode_lr(s, scal, lr);
  if (threadIdx.x == 0) {
    ask = loop_decide_rule(s, scal, lr, status, ftr, ktr, ttr, hw, hs);
    rule = s->next;
  }
  __syncwarp();
  if (!ask) return;
  const int nx = loop_ctrl_choose(s, lr, rule);
  if (threadIdx.x == 0) {
    s->next = nx;
    cudaGraphSetConditional(hs, (unsigned)nx);
    cudaGraphSetConditional(hw, 1u);
  }
}


cudaError_t add_kernel_node(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                            void* func, void** args) {
  cudaKernelNodeParams kp = {};
  kp.func = func;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(32);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

// Capture one branch body into the conditional node's graph; counts its kernels.
template <typename F>
cpals_status capture_into(cpals_ctx* c, cudaGraph_t body, int64_t* count, F&& fn) {
  const int64_t before = c->launches;
  c->ev_used = 0;
  CK(cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cpals_status st = fn();
  cudaGraph_t out = body;
  cudaError_t e = cudaStreamEndCapture(c->stream, &out);
  *count = c->launches - before;
  c->launches = before;
  if (st != CPALS_OK) return st;
  if (e != cudaSuccess) return c->cuda_fail("cudaStreamEndCapture (loop body)", e);
  return CPALS_OK;
}

cpals_status loop_build(cpals_ctx* c, int slot, bool useV) {
  const bool d = is64(c);
  CKS(d ? pp_alloc<double>(c) : pp_alloc<float>(c));
  cudaGraph_t G = nullptr;
  CK(cudaGraphCreate(&G, 0));
  struct Guard {
    cudaGraph_t g;
    ~Guard() { cudaGraphDestroy(g); }
  } guard{G};
  cudaGraphConditionalHandle hw, hs;
  CK(cudaGraphConditionalHandleCreate(&hw, G, 1, cudaGraphCondAssignDefault));
  LoopState* st = static_cast<LoopState*>(c->loop_state);
  const double* scal = c->scal;
  const int* status = c->status;
  cudaGraphNode_t n_init, n_while, n_sw, n_dec;
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  // the while node first (its body holds the switch handle), then the init
  // kernel in front of it
  CK(cudaGraphAddNode(&n_while, G, nullptr, nullptr, 0, &wp));
  cudaGraph_t B = wp.conditional.phGraph_out[0];
  CK(cudaGraphConditionalHandleCreate(&hs, B, 0, 0));
  {
    void* args[] = {&st, &scal, &hw, &hs};
    CK(add_kernel_node(&n_init, G, nullptr, 0, (void*)loop_init_kernel, args));
  }
  CK(cudaGraphAddDependencies(G, &n_init, &n_while, nullptr, 1));
  cudaGraphNodeParams sp = {};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = hs;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = 4;
  CK(cudaGraphAddNode(&n_sw, B, nullptr, nullptr, 0, &sp));
  {
    double* ftr = c->loop_fit;
    int* ktr = c->loop_kind;
    double* ttr = c->loop_time;
    void* args[] = {&st, &scal, &status, &ftr, &ktr, &ttr, &hw, &hs};
    CK(add_kernel_node(&n_dec, B, &n_sw, 1, (void*)loop_decide_kernel, args));
  }
  int64_t* cnt = c->loop_count[slot];
  CKS(capture_into(c, sp.conditional.phGraph_out[0], &cnt[0],
                   [&]() { return d ? als_sweep_launch<double>(c) : als_sweep_launch<float>(c); }));
  CKS(capture_into(c, sp.conditional.phGraph_out[1], &cnt[1], [&]() {
    CKS(d ? pp_build_launch<double>(c) : pp_build_launch<float>(c));
    return d ? pp_sweep_launch<double>(c, useV) : pp_sweep_launch<float>(c, useV);
  }));
  CKS(capture_into(c, sp.conditional.phGraph_out[2], &cnt[2],
                   [&]() { return d ? pp_sweep_launch<double>(c, useV) : pp_sweep_launch<float>(c, useV); }));
  CKS(capture_into(c, sp.conditional.phGraph_out[3], &cnt[3],
                   [&]() { return d ? fitness_launch<double>(c) : fitness_launch<float>(c); }));
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, G, 0);
  if (e != cudaSuccess) return c->cuda_fail("cudaGraphInstantiate (device loop)", e);
  c->loop_exec[slot] = ex;
  return CPALS_OK;
}

// Algorithm 3 with every decision on the device; one synchronisation at the end.
cpals_status run_device_loop(cpals_ctx* c, int max_sweeps, double eps, bool useV, double target,
                             double* fitness_trace, int* kind_trace, double* time_trace, int* n_done,
                             int* reached, bool controlled = false, int* source_trace = nullptr) {
  if (max_sweeps > c->loop_cap) {
    // larger traces: the graphs hold the trace pointers
    for (int i = 0; i < 2; i++)
      if (c->loop_exec[i]) {
        cudaGraphExecDestroy(c->loop_exec[i]);
        c->loop_exec[i] = nullptr;
      }
    if (c->loop_fit) cudaFree(c->loop_fit);
    if (c->loop_time) cudaFree(c->loop_time);
    if (c->loop_kind) cudaFree(c->loop_kind);
    c->loop_fit = c->loop_time = nullptr;
    c->loop_kind = nullptr;
    c->loop_cap = 0;
    const int cap = std::max(1024, max_sweeps);
    CKS(dalloc(c, (void**)&c->loop_fit, (size_t)cap * 8));
    CKS(dalloc(c, (void**)&c->loop_time, (size_t)cap * 8));
    CKS(dalloc(c, (void**)&c->loop_kind, (size_t)cap * 4));
    c->loop_cap = cap;
  }
  if (!c->loop_state) {
    CKS(dalloc(c, &c->loop_state, sizeof(LoopState)));
    if (cudaMallocHost(&c->loop_state_h, sizeof(LoopState)) != cudaSuccess) {
      cudaGetLastError();
      c->loop_state_h = nullptr;
      return c->fail(CPALS_E_OOM, "cudaMallocHost (loop state)");
    }
  }
  const int slot = useV ? 0 : 1;
  if (!c->loop_exec[slot]) CKS(loop_build(c, slot, useV));
  LoopState* h = static_cast<LoopState*>(c->loop_state_h);
  memset(h, 0, sizeof(LoopState));
  h->max_sweeps = max_sweeps;
  h->N = c->N;
  h->eps = eps;
  h->target = target;
  h->tol = c->pp_stop_tol;
  h->ctrl = controlled && c->ctrl_on ? 1 : 0;
  h->conf = c->ctrl_conf;
  h->params = c->ctrl_params;
  CK(cudaMemcpyAsync(c->loop_state, h, sizeof(LoopState), cudaMemcpyHostToDevice, c->stream));
  CK(cudaGraphLaunch(c->loop_exec[slot], c->stream));
  CK(cudaMemcpyAsync(h, c->loop_state, sizeof(LoopState), cudaMemcpyDeviceToHost, c->stream));
  const cpals_status sst = sync_read(c);      // also waits for the copy of the state
  if (sst != CPALS_OK && sst != CPALS_E_TIMEOUT) return sst;
  const int t = std::min(h->t, max_sweeps);
  std::vector<double> ft(t), tt(t);
  std::vector<int> kt(t);
  if (t > 0) {
    CK(cudaMemcpyAsync(ft.data(), c->loop_fit, (size_t)t * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(tt.data(), c->loop_time, (size_t)t * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(kt.data(), c->loop_kind, (size_t)t * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  int64_t l = 1 + ((int64_t)t + h->confirms) + h->confirms * c->loop_count[slot][3];
  for (int i = 0; i < t; i++) {
    const int kind = kt[i] & 0xf;
    l += c->loop_count[slot][kind == CPALS_SWEEP_ALS ? 0 : (kind == CPALS_SWEEP_PP_INIT ? 1 : 2)];
    if (kind == CPALS_SWEEP_PP_INIT) c->ops_built = true;
    if (fitness_trace) fitness_trace[i] = ft[i];
    if (kind_trace) kind_trace[i] = kind;
    if (time_trace) time_trace[i] = tt[i];
    if (source_trace) source_trace[i] = (kt[i] >> 4) & 1;
  }
  c->launches += l;
  if (n_done) *n_done = t;
  if (reached) *reached = h->hit;
  if (sst != CPALS_OK) return sst;
  if (h->err == 3)
    return c->fail(CPALS_E_TIMEOUT, "a bounded device wait gave up during the run");
  if (h->err == 1) return c->fail(CPALS_E_NUMERIC, "non-finite value in a sweep");
  if (h->err == 2) return check_status(c);
  return CPALS_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

cpals_status cpals_create(const int64_t* dims, int N, int R, int precision, cpals_ctx** out) {
  if (!out) return CPALS_E_INVALID;
  *out = nullptr;
  if (!dims || N < 3 || N > kMaxModes || R < 1 || R > kMaxRank) return CPALS_E_INVALID;
  if (precision < CPALS_FP64 || precision > CPALS_MIXED_BF16) return CPALS_E_INVALID;
  for (int i = 0; i < N; i++)
    if (dims[i] < 1 || dims[i] > (1 << 30)) return CPALS_E_INVALID;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return CPALS_E_CUDA;
  }
  if (!(prop.major == 10 && prop.minor == 3)) return CPALS_E_UNSUPPORTED;

  cpals_ctx* c = new cpals_ctx();
  c->dev = dev;
  c->N = N;
  c->R = R;
  c->prec = precision;
  c->total = 1;
  for (int i = 0; i < N; i++) {
    c->dims[i] = dims[i];
    c->total *= dims[i];
    c->smax = std::max<int64_t>(c->smax, dims[i]);
  }
  c->h = (N + 1) / 2;
  for (int i = 0; i < c->h; i++) c->PL *= dims[i];
  for (int i = c->h; i < N; i++) c->PR *= dims[i];
  c->Rpad = (int)cdiv(R, 16) * 16;
  c->esz = precision == CPALS_FP64 ? 8 : 4;
  const size_t esz = c->esz;

  auto bail = [&](cpals_status st) {
    cpals_destroy(c);
    return st;
  };
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return bail(CPALS_E_CUDA);
  for (int i = 0; i < kEvPairs; i++)
    if (cudaEventCreate(&c->ev0[i]) != cudaSuccess || cudaEventCreate(&c->ev1[i]) != cudaSuccess)
      return bail(CPALS_E_CUDA);
  if (setup_small_kernels() != cudaSuccess) return bail(CPALS_E_CUDA);
  if (precision != CPALS_FP64 && setup_df_kernels() != cudaSuccess) return bail(CPALS_E_CUDA);
  if (precision == CPALS_MIXED_BF16 && setup_umma_kernels() != cudaSuccess) return bail(CPALS_E_CUDA);

  cpals_status st = CPALS_OK;
#define AL(ptr, bytes)                                    \
  do {                                                    \
    void* p_ = nullptr;                                   \
    st = dalloc(c, &p_, (bytes));                         \
    if (st != CPALS_OK) return bail(st);                  \
    ptr = decltype(ptr)(p_);                              \
  } while (0)
  AL(c->X, (size_t)c->total * (precision == CPALS_FP64 ? 8 : 4));
  if (precision == CPALS_MIXED_BF16) AL(c->Xb, (size_t)c->total * 2);
  for (int n = 0; n < N; n++) {
    const size_t sR = (size_t)dims[n] * R;
    AL(c->A[n], sR * 8);
    AL(c->Ap[n], sR * 8);
    AL(c->dA[n], sR * 8);
    AL(c->Ac[n], sR * esz);
    AL(c->dAc[n], sR * esz);
  }
  c->dfm = precision != CPALS_FP64;
  if (c->dfm) {
    for (int n = 0; n < N; n++) {
      const size_t sR = (size_t)dims[n] * R;
      AL(c->Alo[n], sR * 4);
      AL(c->Aphi[n], sR * 4);
      AL(c->Aplo[n], sR * 4);
    }
    AL(c->Shi, (size_t)N * R * R * 4);
    AL(c->Slo, (size_t)N * R * R * 4);
    AL(c->Wf, (size_t)N * R * R * 4);
    // padded to 16-byte multiples: the row solve copies them with bulk transfers
    AL(c->Linv, (size_t)R * (R | 1) * 8 + 16);
    AL(c->Gpk, (size_t)R * (R + 1) / 2 * 8 + 16);
    AL(c->Zf, (size_t)R * R * 4 + 16);
  }
  AL(c->S, (size_t)N * R * R * 8);
  AL(c->W, (size_t)N * R * R * 8);
  AL(c->Lf, (size_t)R * R * 8);
  AL(c->Z, (size_t)R * R * 8);
  const int64_t Pmax = std::max(c->PL, c->PR);
  AL(c->ML, (size_t)c->PL * R * esz);
  AL(c->MR, (size_t)c->PR * R * esz);
  AL(c->krp, (size_t)Pmax * R * esz);
  AL(c->tmp[0], (size_t)Pmax * R * esz);
  AL(c->tmp[1], (size_t)Pmax * R * esz);
  AL(c->rhs, (size_t)c->smax * R * esz);
  AL(c->rhs2, (size_t)c->smax * R * 8);
  // split-K partials: enough for 2*152 tiles' worth of outputs of 128 rows
  c->gpart_bytes = std::max<size_t>((size_t)2 * 152 * 128 * R * esz, (size_t)4 * c->smax * R * esz);
  c->gpart_bytes = std::max<size_t>(c->gpart_bytes, (size_t)8 * std::min(c->PL, c->PR) * R * esz);
  // float64 contractions split into about four waves of 64-row tiles
  if (esz == 8) c->gpart_bytes = std::max<size_t>(c->gpart_bytes, (size_t)4 * 3 * 152 * 64 * R * esz);
  AL(c->gpart, c->gpart_bytes);
  if (precision == CPALS_MIXED_BF16) {
    c->Bt_elems = 2 * (size_t)c->Rpad * (size_t)(cdiv(Pmax, 8) * 8);
    AL(c->Bt, c->Bt_elems * 2);
  }
  AL(c->rownorm, (size_t)2 * c->smax * 8);
  AL(c->dscr[0], (size_t)c->smax * R * 8);
  AL(c->dscr[1], (size_t)c->smax * R * 8);
  AL(c->dpart, (size_t)std::max<int64_t>(2 * 152 + 64, cdiv(c->smax, 32) * 26 + 64) * 1024 * 8);
  AL(c->scal, 64 * 8);
  AL(c->status, 4 * sizeof(int));
  AL(c->tickets, 64 * sizeof(int));
  AL(c->umma_sched, 2 * sizeof(int));
  c->umma_err = c->status + 1;
#undef AL
  if (cudaMallocHost((void**)&c->scal_h, 64 * 8) != cudaSuccess ||
      cudaMallocHost((void**)&c->status_h, 4 * sizeof(int)) != cudaSuccess)
    return bail(CPALS_E_OOM);
  if (cudaMemset(c->scal, 0, 64 * 8) != cudaSuccess || cudaMemset(c->status, 0, 16) != cudaSuccess ||
      cudaMemset(c->tickets, 0, 64 * sizeof(int)) != cudaSuccess ||
      cudaMemset(c->umma_sched, 0, 2 * sizeof(int)) != cudaSuccess ||
      cudaMemset(c->W, 0, (size_t)N * R * R * 8) != cudaSuccess)
    return bail(CPALS_E_CUDA);
  memset(c->scal_h, 0, 64 * 8);
  *out = c;
  return CPALS_OK;
}

void cpals_destroy(cpals_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);
  drop_graphs(c);
  auto F = [](void* p) {
    if (p) cudaFree(p);
  };
  F(c->X);
  F(c->Xb);
  for (int n = 0; n < kMaxModes; n++) {
    F(c->A[n]); F(c->Ap[n]); F(c->dA[n]); F(c->Ac[n]); F(c->dAc[n]); F(c->Mp[n]);
    for (int m = 0; m < kMaxModes; m++) F(c->ops[n][m]);
    F(c->Alo[n]); F(c->Aphi[n]); F(c->Aplo[n]);
  }
  for (void* p : c->lvl_bufs) F(p);
  F(c->Shi); F(c->Slo); F(c->Wf); F(c->Linv); F(c->Gpk); F(c->Zf);
  F(c->S); F(c->W); F(c->Lf); F(c->Z); F(c->ML); F(c->MR); F(c->krp); F(c->tmp[0]); F(c->tmp[1]);
  F(c->rhs); F(c->rhs2); F(c->gpart); F(c->Bt); F(c->rownorm); F(c->dpart); F(c->scal);
  F(c->status); F(c->tickets); F(c->umma_sched); F(c->dscr[0]); F(c->dscr[1]);
  F(c->ctrl_params); F(c->ctrl_io);
  if (c->ctrl_io_h) cudaFreeHost(c->ctrl_io_h);
  for (void* p : c->snap_bufs) F(p);
  F(c->loop_state); F(c->loop_fit); F(c->loop_time); F(c->loop_kind);
  if (c->loop_state_h) cudaFreeHost(c->loop_state_h);
  if (c->scal_h) cudaFreeHost(c->scal_h);
  if (c->status_h) cudaFreeHost(c->status_h);
  for (int i = 0; i < kEvPairs; i++) {
    if (c->ev0[i]) cudaEventDestroy(c->ev0[i]);
    if (c->ev1[i]) cudaEventDestroy(c->ev1[i]);
  }
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

cpals_status cpals_set_stream(cpals_ctx* c, void* stream) {
  if (!c) return CPALS_E_INVALID;
  c->user = (cudaStream_t)stream;
  return CPALS_OK;
}

// Many independent decompositions (tensors of different shapes, each with its
// own context): worker threads take the next context from a shared counter
// and run Algorithm 3 on it (cpals_run, on the context's own streams), so up
// to `workers` decompositions are in flight on the GPU at once while each
// keeps its own controller.  Uneven instances balance themselves; the result
// of every instance is the one cpals_run gives it alone.
cpals_status cpals_run_batch(cpals_ctx* const* ctxs, int n, int workers, int max_sweeps, double eps,
                             int use_V, const double* targets, double* fitness_out,
                             int* sweeps_out, int* status_out) {
  if (!ctxs || n < 0 || workers < 1 || max_sweeps < 1) return CPALS_E_INVALID;
  for (int i = 0; i < n; i++)
    if (!ctxs[i]) return CPALS_E_INVALID;
  // operator buffers before any worker captures a graph
  for (int i = 0; i < n; i++) {
    cpals_ctx* c = ctxs[i];
    if (cudaSetDevice(c->dev) != cudaSuccess) return c->cuda_fail("cudaSetDevice", cudaGetLastError());
    CKS(is64(c) ? pp_alloc<double>(c) : pp_alloc<float>(c));
  }
  std::atomic<int> next{0};
  auto work = [&]() {
    std::vector<double> ft((size_t)max_sweeps);
    while (true) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      cpals_ctx* c = ctxs[i];
      int nd = 0, rc = 0;
      cpals_status st = cudaSetDevice(c->dev) == cudaSuccess ? CPALS_OK : CPALS_E_CUDA;
      if (st == CPALS_OK)
        st = cpals_run(c, max_sweeps, eps, use_V, targets ? targets[i] : 0.0, ft.data(), nullptr,
                       nullptr, &nd, &rc);
      if (fitness_out) fitness_out[i] = nd > 0 ? ft[nd - 1] : std::nan("");
      if (sweeps_out) sweeps_out[i] = nd;
      if (status_out) status_out[i] = (int)st;
    }
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < std::min(workers, n); w++) pool.emplace_back(work);
  for (auto& t : pool) t.join();
  return CPALS_OK;
}

const char* cpals_last_error(const cpals_ctx* c) { return c ? c->err.c_str() : "null context"; }

cpals_status cpals_set_tensor(cpals_ctx* c, const void* data, int dtype, int on_device) {
  if (!c || !data || (dtype != 0 && dtype != 1)) return c ? c->fail(CPALS_E_INVALID, "bad tensor argument") : CPALS_E_INVALID;
  Join j(c);
  const int64_t n = c->total;
  const size_t insz = dtype == 0 ? 8 : 4;
  const bool store64 = c->prec == CPALS_FP64;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if ((dtype == 0) == store64) {
    CK(cudaMemcpyAsync(c->X, data, n * insz, kind, c->stream));
  } else {
    void* tmp = nullptr;
    CKS(dalloc(c, &tmp, n * insz));
    cudaError_t e = cudaMemcpyAsync(tmp, data, n * insz, kind, c->stream);
    if (e == cudaSuccess) {
      if (dtype == 0) convert<double, float>((const double*)tmp, (float*)c->X, n, c->L());
      else convert<float, double>((const float*)tmp, (double*)c->X, n, c->L());
      e = cudaStreamSynchronize(c->stream);
    }
    cudaFree(tmp);
    if (e != cudaSuccess) return c->cuda_fail("set_tensor copy", e);
  }
  if (c->prec == CPALS_MIXED_BF16) convert<float, __nv_bfloat16>((const float*)c->X, c->Xb, n, c->L());
  if (store64) sumsq<double>((const double*)c->X, n, c->dpart, c->scal + 40, c->L());
  else sumsq<float>((const float*)c->X, n, c->dpart, c->scal + 40, c->L());
  double nx = 0;
  CK(cudaMemcpyAsync(&nx, c->scal + 40, 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  c->normX2 = nx;
  c->have_tensor = true;
  c->ops_built = false;
  // the captured graphs stay valid: the fitness kernels read ||X||^2 from
  // device memory (scal[40]) when they run
  return CPALS_OK;
}

cpals_status cpals_init_factors(cpals_ctx* c, const double* const* factors) {
  if (!c || !factors) return c ? c->fail(CPALS_E_INVALID, "factors is NULL") : CPALS_E_INVALID;
  for (int n = 0; n < c->N; n++)
    if (!factors[n]) return c->fail(CPALS_E_INVALID, "factor pointer is NULL");
  Join j(c);
  const int R = c->R;
  CK(cudaMemsetAsync(c->status, 0, 16, c->stream));
  for (int n = 0; n < c->N; n++) {
    const int64_t sR = c->dims[n] * R;
    // a tied mode starts from its partner's factor (Sec. 5.1)
    const double* src = factors[tied(c, n) ? c->tie[n] : n];
    CK(cudaMemcpyAsync(c->A[n], src, sR * 8, cudaMemcpyHostToDevice, c->stream));
    // the start of Algorithm 3: dA <- A, S <- A^T A
    CK(cudaMemcpyAsync(c->dA[n], c->A[n], sR * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (is64(c)) {
      convert<double, double>(c->A[n], P<double>(c->Ac[n]), sR, c->L());
      convert<double, double>(c->A[n], P<double>(c->dAc[n]), sR, c->L());
    } else {
      convert<double, float>(c->A[n], P<float>(c->Ac[n]), sR, c->L());
      convert<double, float>(c->A[n], P<float>(c->dAc[n]), sR, c->L());
    }
    sumsq<double>(c->A[n], sR, c->dpart, c->scal + 8 + 2 * n, c->L());
    CK(cudaMemcpyAsync(c->scal + 9 + 2 * n, c->scal + 8 + 2 * n, 8, cudaMemcpyDeviceToDevice, c->stream));
    // rownorm is not needed: the Gram kernel reduces it into a scratch slot
    CK(cudaMemsetAsync(c->rownorm, 0, 2 * c->dims[n] * 8, c->stream));
    const int64_t off = (int64_t)n * R * R;
    if (c->dfm) {
      split_df(c->A[n], P<float>(c->Ac[n]), c->Alo[n], sR, c->L());
      gram_df(P<const float>(c->Ac[n]), c->Alo[n], P<const float>(c->Ac[n]),
              P<const float>(c->dAc[n]), c->S + off, c->Shi + off, c->Slo + off, c->Wf + off,
              false, (int)c->dims[n], R, (const float2*)c->rownorm, c->scal + 48, c->Shi,
              c->Slo, c->N, n, (n + 1) % c->N, c->Gpk, c->L());
    } else {
      gram_update<double>(c->A[n], P<const double>(c->Ac[n]), P<const double>(c->dAc[n]),
                          c->S + off, c->W + off, false, (int)c->dims[n], R, c->rownorm,
                          c->scal + 48, c->dpart, c->tickets, c->L());
    }
  }
  if (c->dfm) CK(cudaMemsetAsync(c->Wf, 0, (size_t)c->N * R * R * 4, c->stream));
  CK(cudaMemsetAsync(c->W, 0, (size_t)c->N * R * R * 8, c->stream));
  CKS(sync_read(c));
  c->have_factors = true;
  c->ops_built = false;
  return CPALS_OK;
}

cpals_status cpals_als_sweep(cpals_ctx* c, double* fitness_out) {
  CKS(ready(c));
  Join j(c);
  CKS(do_als(c));
  CKS(sync_read(c));
  if (fitness_out) *fitness_out = c->scal_h[0];
  return check_status(c);
}

cpals_status cpals_pp_build_operators(cpals_ctx* c) {
  CKS(ready(c));
  Join j(c);
  CKS(do_build(c));
  CKS(sync_read(c));
  c->ops_built = true;
  return CPALS_OK;
}

cpals_status cpals_pp_sweep(cpals_ctx* c, int use_V, double* fitness_out) {
  CKS(ready(c));
  if (!c->ops_built) return c->fail(CPALS_E_STATE, "PP operators not built: call cpals_pp_build_operators");
  Join j(c);
  CKS(do_pp(c, use_V != 0));
  CKS(sync_read(c));
  if (fitness_out) *fitness_out = c->scal_h[0];
  return check_status(c);
}

cpals_status cpals_fitness(cpals_ctx* c, double* out) {
  CKS(ready(c));
  if (!out) return c->fail(CPALS_E_INVALID, "out is NULL");
  Join j(c);
  CKS(do_fit(c));
  CKS(sync_read(c));
  *out = c->scal_h[0];
  return CPALS_OK;
}

cpals_status cpals_get_factors(cpals_ctx* c, double* const* out) {
  CKS(ready(c));
  if (!out) return c->fail(CPALS_E_INVALID, "out is NULL");
  Join j(c);
  for (int n = 0; n < c->N; n++) {
    if (!out[n]) return c->fail(CPALS_E_INVALID, "out[n] is NULL");
    CK(cudaMemcpyAsync(out[n], c->A[n], c->dims[n] * c->R * 8, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return CPALS_OK;
}

cpals_status cpals_get_dA_ratios(cpals_ctx* c, double* out) {
  CKS(ready(c));
  if (!out) return c->fail(CPALS_E_INVALID, "out is NULL");
  Join j(c);
  CKS(sync_read(c));
  for (int n = 0; n < c->N; n++)
    out[n] = std::sqrt(c->scal_h[8 + 2 * n]) / std::sqrt(c->scal_h[9 + 2 * n]);
  return CPALS_OK;
}

cpals_status cpals_pinv_modes(cpals_ctx* c, int* mask) {
  if (!c || !mask) return CPALS_E_INVALID;
  Join j(c);
  CKS(sync_read(c));
  *mask = (c->status_h[0] >> 16) & 0xffff;
  return CPALS_OK;
}

cpals_status cpals_run(cpals_ctx* c, int max_sweeps, double eps, int use_V, double target,
                       double* fitness_trace, int* kind_trace, double* time_trace, int* n_done,
                       int* reached) {
  CKS(ready(c));
  if (max_sweeps < 0) return c->fail(CPALS_E_INVALID, "max_sweeps < 0");
  Join j(c);
  if (c->device_loop && c->graphs && !c->profiling && max_sweeps > 0) {
    if (c->loop_note.empty()) {
      const std::string saved = c->err;
      cpals_status st = run_device_loop(c, max_sweeps, eps, use_V != 0, target, fitness_trace,
                                        kind_trace, time_trace, n_done, reached);
      // a graph this driver cannot build or run with conditional nodes: the
      // host loop below takes over (the reason stays in loop_note)
      if (st != CPALS_E_CUDA || c->loop_exec[use_V ? 0 : 1]) return st;
      c->loop_note = c->err;
      c->err = saved;
      cudaGetLastError();
    }
  }
  const auto t0 = std::chrono::steady_clock::now();
  int t = 0;
  int hit = 0;
  double f_last = -1e300, f_prev = -1e300;   // fitness seen after the last two sweeps
  int in_run = 0;                              // PP sweeps of the current PP run
  auto record = [&](int kind, double f) {
    if (fitness_trace) fitness_trace[t] = f;
    if (kind_trace) kind_trace[t] = kind;
    if (time_trace)
      time_trace[t] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    t++;
    f_prev = f_last;
    f_last = f;
    in_run = kind == CPALS_SWEEP_ALS ? 0 : (kind == CPALS_SWEEP_PP_INIT ? 1 : in_run + 1);
  };
  const double tol = c->pp_stop_tol;
  auto gained = [&]() { return !(tol > 0.0) || in_run < 2 || f_last - f_prev >= tol; };
  cpals_status st = CPALS_OK;
  // make sure the eps test sees current ratios
  st = sync_read(c);
  while (st == CPALS_OK && t < max_sweeps && !hit) {
    if (eps > 0 && all_small(c, eps)) {
      st = do_build(c);
      if (st != CPALS_OK) break;
      c->ops_built = true;
      st = sync_read(c);
      bool first = true;
      while (st == CPALS_OK && t < max_sweeps && all_small(c, eps) && (first || gained())) {
        st = do_pp(c, use_V != 0);
        if (st != CPALS_OK) break;
        st = sync_read(c);
        if (st != CPALS_OK) break;
        st = check_status(c);
        double f = c->scal_h[0];
        if (target > 0 && f >= target) {
          // confirm with the exact fitness (Sec. 5)
          st = do_fit(c);
          if (st == CPALS_OK) st = sync_read(c);
          if (st == CPALS_OK && c->scal_h[0] >= target) {
            f = c->scal_h[0];
            hit = 1;
          }
        }
        record(first ? CPALS_SWEEP_PP_INIT : CPALS_SWEEP_PP_APPROX, f);
        first = false;
        if (hit) break;
      }
      if (st != CPALS_OK || hit || t >= max_sweeps) break;
    }
    st = do_als(c);
    if (st != CPALS_OK) break;
    st = sync_read(c);
    if (st != CPALS_OK) break;
    st = check_status(c);
    const double f = c->scal_h[0];
    if (target > 0 && f >= target) hit = 1;
    record(CPALS_SWEEP_ALS, f);
  }
  if (n_done) *n_done = t;
  if (reached) *reached = hit;
  return st;
}

cpals_status cpals_set_controller(cpals_ctx* c, const float* params, int nparams, double confidence) {
  if (!c) return CPALS_E_INVALID;
  if (!params) {
    c->ctrl_on = false;
    return CPALS_OK;
  }
  if (nparams != ctrl_param_count(kCtrlFeatures) || !(confidence >= 0.0 && confidence <= 1.0))
    return c->fail(CPALS_E_INVALID, "controller: need " + std::to_string(ctrl_param_count(kCtrlFeatures)) +
                                        " parameters and 0 <= confidence <= 1");
  if (!c->ctrl_params) CKS(dalloc(c, (void**)&c->ctrl_params, (size_t)nparams * 4));
  if (!c->ctrl_io) CKS(dalloc(c, (void**)&c->ctrl_io, 64 * 4));
  if (!c->ctrl_io_h) CK(cudaMallocHost(&c->ctrl_io_h, 64 * 4));
  CK(cudaMemcpyAsync(c->ctrl_params, params, (size_t)nparams * 4, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->ctrl_conf = confidence;
  c->ctrl_on = true;
  return CPALS_OK;
}

cpals_status cpals_run_controlled(cpals_ctx* c, int max_sweeps, double eps, int use_V, double target,
                                  double* fitness_trace, int* kind_trace, double* time_trace,
                                  int* source_trace, int* n_done, int* reached) {
  CKS(ready(c));
  if (max_sweeps < 0 || !(eps > 0)) return c->fail(CPALS_E_INVALID, "max_sweeps < 0 or eps <= 0");
  Join j(c);
  if (c->device_loop && c->graphs && !c->profiling && max_sweeps > 0 && c->loop_note.empty()) {
    // the decisions inside the device loop's graph (features, forward pass
    // and rule in its decide kernel): no host round trip per sweep
    const std::string saved = c->err;
    cpals_status st = run_device_loop(c, max_sweeps, eps, use_V != 0, target, fitness_trace, kind_trace,
                                      time_trace, n_done, reached, true, source_trace);
    c->ctrl_last_dev = true;
    if (st != CPALS_E_CUDA || c->loop_exec[use_V ? 0 : 1]) return st;
    c->loop_note = c->err;
    c->err = saved;
    cudaGetLastError();
  }
  c->ctrl_last_dev = false;
  const auto t0 = std::chrono::steady_clock::now();
  CtrlHist h;
  int t = 0, hit = 0;
  double f_last = -1e300, f_prev = -1e300;     // fitness seen after the last two sweeps
  int in_run = 0;                                // PP sweeps of the current PP run
  const double tol = c->pp_stop_tol;
  cpals_status st = sync_read(c);
  // the current state: after cpals_init_factors dA = A, so the first sweep is exact
  h.res[0] = 1.0 - c->scal_h[0];
  while (st == CPALS_OK && t < max_sweeps && !hit) {
    // the paper's eps rule (Algorithm 3): stay in / enter the PP phase while
    // every ||dA|| < eps ||A|| (and, with a stopping tolerance, while the PP
    // run still gains, as in cpals_run)
    const bool small = all_small(c, eps);
    const bool gain = !(tol > 0.0) || in_run < 2 || f_last - f_prev >= tol;
    const int rule = h.pp_ready ? ((small && gain) ? ACT_PP : ACT_ALS) : (small ? ACT_REBUILD : ACT_ALS);
    int act = rule, src = 0;
    if (c->ctrl_on) {
      ctrl_features(c, h, eps, c->ctrl_io_h);
      CK(cudaMemcpyAsync(c->ctrl_io, c->ctrl_io_h, kCtrlFeatures * 4, cudaMemcpyHostToDevice, c->stream));
      mlp_forward(c->ctrl_params, kCtrlFeatures, c->ctrl_io, 1, c->ctrl_io + 32, c->L());
      CK(cudaMemcpyAsync(c->ctrl_io_h + 32, c->ctrl_io + 32, kCtrlClasses * 4, cudaMemcpyDeviceToHost,
                         c->stream));
      CK(cudaStreamSynchronize(c->stream));
      const float* pr = c->ctrl_io_h + 32;
      int best = 0;
      for (int k = 1; k < kCtrlClasses; k++)
        if (pr[k] > pr[best]) best = k;
      // the rule stands in when the network is unsure or asks for a PP sweep
      // without valid operators
      if (pr[best] >= c->ctrl_conf && !(best == ACT_PP && !h.pp_ready)) {
        act = best;
        src = 1;
      }
    }
    st = do_action(c, act, use_V != 0);
    if (st != CPALS_OK) break;
    double f = c->scal_h[0];
    if (act != ACT_ALS && target > 0 && f >= target) {
      // a PP estimate reached the target: confirm with the exact fitness (Sec. 5)
      st = exact_fitness(c, &f);
      if (st != CPALS_OK) break;
    }
    if (target > 0 && f >= target) hit = 1;
    h.push(c, act, f);
    f_prev = f_last;
    f_last = f;
    in_run = act == ACT_ALS ? 0 : (act == ACT_REBUILD ? 1 : in_run + 1);
    if (fitness_trace) fitness_trace[t] = f;
    if (kind_trace)
      kind_trace[t] = act == ACT_ALS ? CPALS_SWEEP_ALS : act == ACT_REBUILD ? CPALS_SWEEP_PP_INIT : CPALS_SWEEP_PP_APPROX;
    if (time_trace)
      time_trace[t] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (source_trace) source_trace[t] = src;
    t++;
  }
  if (n_done) *n_done = t;
  if (reached) *reached = hit;
  return st;
}

cpals_status cpals_controller_last(const cpals_ctx* c, float* features, float* probs) {
  if (!c) return CPALS_E_INVALID;
  const float* x = nullptr;
  const float* p = nullptr;
  if (c->ctrl_last_dev && c->loop_state_h) {
    const LoopState* h = static_cast<const LoopState*>(c->loop_state_h);
    x = h->last_x;
    p = h->last_p;
  } else if (c->ctrl_io_h) {
    x = c->ctrl_io_h;
    p = c->ctrl_io_h + 32;
  } else {
    return CPALS_E_STATE;
  }
  if (features) memcpy(features, x, kCtrlFeatures * sizeof(float));
  if (probs) memcpy(probs, p, kCtrlClasses * sizeof(float));
  return CPALS_OK;
}

cpals_status cpals_set_controller_labels(cpals_ctx* c, double target, int max_rollout) {
  if (!c) return CPALS_E_INVALID;
  if (!(target >= 0.0) || (target > 0.0 && max_rollout < 1))
    return c->fail(CPALS_E_INVALID, "controller labels: target >= 0 and, with a target, max_rollout >= 1");
  c->label_target = target;
  c->label_rollout = max_rollout;
  return CPALS_OK;
}

cpals_status cpals_controller_log(cpals_ctx* c, int steps, double eps, int use_V, float* features,
                                  int* labels, double* gains, double* costs, int* n_out) {
  CKS(ready(c));
  if (steps < 0 || !(eps > 0) || !features || !labels || !gains || !costs || !n_out)
    return c->fail(CPALS_E_INVALID, "bad argument");
  Join j(c);
  CtrlHist h;
  cpals_status st = sync_read(c);
  h.res[0] = 1.0 - c->scal_h[0];
  int t = 0;
  auto now = [] { return std::chrono::steady_clock::now(); };
  while (st == CPALS_OK && t < steps) {
    double f0 = 0;
    st = exact_fitness(c, &f0);
    if (st != CPALS_OK) break;
    if (c->label_target > 0.0 && f0 >= c->label_target) break;   // the trajectory is at the target
    ctrl_features(c, h, eps, features + (size_t)t * kCtrlFeatures);
    // candidates: a PP sweep when one is possible, else rebuild + PP sweep,
    // against an ALS sweep
    const int cand[2] = {h.pp_ready ? ACT_PP : ACT_REBUILD, ACT_ALS};
    const bool to_target = c->label_target > 0.0;
    double rate[3] = {-1e300, -1e300, -1e300};
    double ttt[3] = {1e300, 1e300, 1e300};     // time to the target (to_target)
    double fend[3] = {-1e300, -1e300, -1e300};  // exact fitness at the end of the trial
    for (int k = 0; k < 3; k++) {
      gains[(size_t)t * 3 + k] = std::nan("");
      costs[(size_t)t * 3 + k] = std::nan("");
    }
    // a trial to the target may rebuild the operators later on: save them too
    st = snapshot_take(c, to_target || cand[0] == ACT_REBUILD);
    for (int k = 0; k < 2 && st == CPALS_OK; k++) {
      if (k > 0) st = snapshot_restore(c);
      if (st != CPALS_OK) break;
      CK(cudaStreamSynchronize(c->stream));
      const auto ta = now();
      bool hit = false;
      if (to_target) {
        // the candidate, then Algorithm 3's rule (as the host loop of
        // cpals_run) until the target or label_rollout sweeps
        int act = cand[k], in_run = 0;
        double fl = -1e300, fp = -1e300;
        const double tol = c->pp_stop_tol;
        for (int d = 0; d < c->label_rollout && st == CPALS_OK; d++) {
          st = do_action(c, act, use_V != 0);
          if (st != CPALS_OK) break;
          double f = c->scal_h[0];
          if (act != ACT_ALS && f >= c->label_target) st = exact_fitness(c, &f);   // confirm (Sec. 5)
          if (st != CPALS_OK) break;
          if (f >= c->label_target) {
            hit = true;
            break;
          }
          in_run = act == ACT_ALS ? 0 : (act == ACT_REBUILD ? 1 : in_run + 1);
          fp = fl;
          fl = f;
          const bool small = all_small(c, eps);
          const bool gain = !(tol > 0.0) || in_run < 2 || fl - fp >= tol;
          act = act == ACT_ALS ? (small ? ACT_REBUILD : ACT_ALS) : (small && gain ? ACT_PP : ACT_ALS);
        }
      } else {
        // kCtrlHorizon sweeps of the candidate's kind (a horizon of several
        // sweeps lifts the gains above the rounding of the fitness)
        for (int d = 0; d < kCtrlHorizon && st == CPALS_OK; d++)
          st = do_action(c, d == 0 ? cand[k] : (cand[k] == ACT_ALS ? ACT_ALS : ACT_PP), use_V != 0);
      }
      const double dt = std::chrono::duration<double>(now() - ta).count();
      if (st == CPALS_E_SINGULAR || st == CPALS_E_NUMERIC) {
        // a trial that breaks down (a non-finite Gamma, factor or fitness:
        // approximated sweeps can diverge) loses; the next trial and the
        // labelled action start from the snapshot
        st = CPALS_OK;
        continue;
      }
      double f = 0;
      if (st == CPALS_OK) st = exact_fitness(c, &f);
      if (st != CPALS_OK) break;
      gains[(size_t)t * 3 + cand[k]] = f - f0;
      costs[(size_t)t * 3 + cand[k]] = dt;
      rate[cand[k]] = (f - f0) / std::max(dt, 1e-9);
      fend[cand[k]] = f;
      if (hit) ttt[cand[k]] = dt;
    }
    if (st != CPALS_OK) break;
    int label;
    if (to_target) {
      // the shorter time to the target; if neither trial reached it, the
      // higher fitness at the end of the trial (ties to the exact sweep)
      const bool any = ttt[cand[0]] < 1e300 || ttt[ACT_ALS] < 1e300;
      label = any ? (ttt[cand[0]] < ttt[ACT_ALS] ? cand[0] : ACT_ALS)
                  : (fend[cand[0]] > fend[ACT_ALS] ? cand[0] : ACT_ALS);
    } else {
      // the larger fitness gain per second (ties and breakdowns of the PP
      // candidate to the exact sweep)
      label = rate[cand[0]] > rate[ACT_ALS] && gains[(size_t)t * 3 + cand[0]] > 0 ? cand[0] : ACT_ALS;
    }
    labels[t] = label;
    // continue the trajectory with the labelled action
    st = snapshot_restore(c);
    if (st == CPALS_OK) st = do_action(c, label, use_V != 0);
    if (st != CPALS_OK) break;
    h.push(c, label, c->scal_h[0]);
    t++;
  }
  *n_out = t;
  return st;
}

cpals_status cpals_mlp_forward(const float* params, int nparams, const float* X, int n, float* probs) {
  if (!params || !X || !probs || n < 0 || nparams != ctrl_param_count(kCtrlFeatures)) return CPALS_E_INVALID;
  if (n == 0) return CPALS_OK;
  float *dp = nullptr, *dx = nullptr, *dpr = nullptr;
  int64_t cnt = 0;
  auto done = [&](cpals_status s) {
    cudaFree(dp);
    cudaFree(dx);
    cudaFree(dpr);
    return s;
  };
  if (cudaMalloc(&dp, (size_t)nparams * 4) != cudaSuccess || cudaMalloc(&dx, (size_t)n * kCtrlFeatures * 4) != cudaSuccess ||
      cudaMalloc(&dpr, (size_t)n * kCtrlClasses * 4) != cudaSuccess) {
    cudaGetLastError();
    return done(CPALS_E_OOM);
  }
  if (cudaMemcpy(dp, params, (size_t)nparams * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dx, X, (size_t)n * kCtrlFeatures * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return done(CPALS_E_CUDA);
  mlp_forward(dp, kCtrlFeatures, dx, n, dpr, Launch{0, &cnt});
  if (cudaMemcpy(probs, dpr, (size_t)n * kCtrlClasses * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return done(CPALS_E_CUDA);
  return done(CPALS_OK);
}

cpals_status cpals_mlp_train(const float* X, const int* y, const float* w, int n, float* params,
                             int nparams, int epochs, double lr, double decay, double* loss_out) {
  if (!X || !y || !w || !params || n < 1 || epochs < 0 || nparams != ctrl_param_count(kCtrlFeatures) ||
      !(lr > 0))
    return CPALS_E_INVALID;
  for (int i = 0; i < n; i++)
    if (y[i] < 0 || y[i] >= kCtrlClasses || !(w[i] >= 0)) return CPALS_E_INVALID;
  double wsum = 0;
  for (int i = 0; i < n; i++) wsum += w[i];
  if (!(wsum > 0)) return CPALS_E_INVALID;
  const int F = kCtrlFeatures;
  std::vector<void*> bufs;
  auto al = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    bufs.push_back(p);
    return p;
  };
  auto done = [&](cpals_status s) {
    for (void* p : bufs) cudaFree(p);
    return s;
  };
  float* dp = (float*)al((size_t)nparams * 4);
  float* dm = (float*)al((size_t)nparams * 4);
  float* dv = (float*)al((size_t)nparams * 4);
  float* dx = (float*)al((size_t)n * F * 4);
  int* dy = (int*)al((size_t)n * 4);
  float* dw = (float*)al((size_t)n * 4);
  float* hs = (float*)al((size_t)n * kCtrlHidden * 4);
  float* dz = (float*)al((size_t)n * kCtrlClasses * 4);
  float* dh = (float*)al((size_t)n * kCtrlHidden * 4);
  float* dl = (float*)al((size_t)n * 4);
  if (!dp || !dm || !dv || !dx || !dy || !dw || !hs || !dz || !dh || !dl) return done(CPALS_E_OOM);
  if (cudaMemcpy(dp, params, (size_t)nparams * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dx, X, (size_t)n * F * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dy, y, (size_t)n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dw, w, (size_t)n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(dm, 0, (size_t)nparams * 4) != cudaSuccess || cudaMemset(dv, 0, (size_t)nparams * 4) != cudaSuccess)
    return done(CPALS_E_CUDA);
  int64_t cnt = 0;
  for (int e = 1; e <= epochs; e++)
    mlp_train_epoch(dp, dm, dv, F, dx, dy, dw, n, (float)(1.0 / wsum), (float)lr, (float)decay, e, hs, dz,
                    dh, dl, Launch{0, &cnt});
  if (cudaMemcpy(params, dp, (size_t)nparams * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return done(CPALS_E_CUDA);
  if (loss_out) {
    // loss of the final parameters: one more forward/backward pass
    if (epochs > 0) {
      mlp_train_epoch(dp, dm, dv, F, dx, dy, dw, n, 0.f, 0.f, 0.f, epochs + 1, hs, dz, dh, dl, Launch{0, &cnt});
    } else {
      mlp_train_epoch(dp, dm, dv, F, dx, dy, dw, n, 0.f, 0.f, 0.f, 1, hs, dz, dh, dl, Launch{0, &cnt});
    }
    std::vector<float> hl(n);
    if (cudaMemcpy(hl.data(), dl, (size_t)n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return done(CPALS_E_CUDA);
    double sl = 0;
    for (int i = 0; i < n; i++) sl += hl[i];
    *loss_out = sl / wsum;
  }
  if (cudaGetLastError() != cudaSuccess) return done(CPALS_E_CUDA);
  return done(CPALS_OK);
}

cpals_status cpals_mttkrp(cpals_ctx* c, int n, double* out) {
  CKS(ready(c));
  if (n < 0 || n >= c->N || !out) return c->fail(CPALS_E_INVALID, "bad mode or NULL out");
  Join j(c);
  c->ev_used = 0;
  const int64_t cnt = c->dims[n] * c->R;
  if (is64(c)) {
    const double* r = nullptr;
    CKS(mttkrp_launch<double>(c, n, &r));
    CKS(sync_read(c));
    return copy_out<double>(c, r, cnt, out);
  }
  const float* r = nullptr;
  CKS(mttkrp_launch<float>(c, n, &r));
  CKS(sync_read(c));
  return copy_out<float>(c, r, cnt, out);
}

cpals_status cpals_get_operator(cpals_ctx* c, int i, int n, double* out) {
  CKS(ready(c));
  if (!c->ops_built) return c->fail(CPALS_E_STATE, "PP operators not built");
  if (i < 0 || n < 0 || i >= c->N || n >= c->N || i > n || !out)
    return c->fail(CPALS_E_INVALID, "need 0 <= i <= n < N");
  Join j(c);
  const void* src = i == n ? c->Mp[n] : c->ops[i][n];
  const int64_t cnt = (i == n ? 1 : c->dims[i]) * c->dims[n] * c->R;
  if (is64(c)) return copy_out<double>(c, (const double*)src, cnt, out);
  return copy_out<float>(c, (const float*)src, cnt, out);
}

cpals_status cpals_pp_mttkrp(cpals_ctx* c, int n, int use_V, double* out) {
  CKS(ready(c));
  if (!c->ops_built) return c->fail(CPALS_E_STATE, "PP operators not built");
  if (n < 0 || n >= c->N || !out) return c->fail(CPALS_E_INVALID, "bad mode or NULL out");
  Join j(c);
  c->ev_used = 0;
  const int R = c->R;
  const int s = (int)c->dims[n];
  const int64_t cnt = (int64_t)s * R;
  auto go = [&](auto tag) -> cpals_status {
    using T = decltype(tag);
    PPTerm<T> terms[kMaxModes];
    pp_terms<T>(c, n, terms);
    pp_correct<T>(P<const T>(c->Mp[n]), terms, c->N - 1, P<T>(c->rhs), s, R, c->L());
    const T* res = P<const T>(c->rhs);
    if (use_V) {
      if (c->dfm) {
        chol_df(c->Shi, c->Slo, c->Wf, nullptr, c->N, n, R, c->Linv, c->Zf, true, c->status, c->L());
        convert<float, double>(c->Zf, c->Z, (int64_t)R * R, c->L());
      } else {
        gamma_chol(c->S, c->W, c->N, n, R, c->Lf, c->Z, true, c->status, c->L());
      }
      vterm<T>(P<const T>(c->rhs), P<const T>(c->Ac[n]), c->Z, P<T>(c->rhs2), s, R, c->L());
      CKS(sync_read(c));
      return copy_out<T>(c, P<const T>(c->rhs2), cnt, out);
    }
    CKS(sync_read(c));
    return copy_out<T>(c, res, cnt, out);
    return CPALS_OK;
  };
  return is64(c) ? go(double{}) : go(float{});
}

cpals_status cpals_normal_solve(cpals_ctx* c, int n, const double* rhs, double* out) {
  CKS(ready(c));
  if (n < 0 || n >= c->N || !rhs || !out) return c->fail(CPALS_E_INVALID, "bad mode or NULL buffer");
  Join j(c);
  const int R = c->R;
  const int s = (int)c->dims[n];
  const int64_t cnt = (int64_t)s * R;
  CK(cudaMemsetAsync(c->status, 0, 16, c->stream));
  CK(cudaMemcpyAsync(c->dscr[0], rhs, cnt * 8, cudaMemcpyHostToDevice, c->stream));
  // scratch: dscr[1] <- A_new (float64); the other outputs of the row solve go to
  // rhs2 (s*R*8 bytes), tmp[0] and dscr[0] (the rhs is consumed first)
  if (c->dfm) {
    float* frhs = P<float>(c->rhs);
    convert<double, float>(c->dscr[0], frhs, cnt, c->L());
    chol_df(c->Shi, c->Slo, c->Wf, nullptr, c->N, n, R, c->Linv, c->Zf, false, c->status, c->L());
    float* hi = P<float>(c->rhs2);
    float* lo = hi + cnt;
    CK(cudaMemsetAsync(hi, 0, cnt * 8, c->stream));
    solve_df(frhs, c->dscr[1], hi, lo, nullptr, nullptr, c->dscr[0], P<float>(c->tmp[0]), c->Linv,
             nullptr, (float2*)c->rownorm, s, R, n, 1.0, c->status, c->L());
  } else {
    gamma_chol(c->S, c->W, c->N, n, R, c->Lf, c->Z, false, c->status, c->L());
    CK(cudaMemsetAsync(c->dscr[1], 0, cnt * 8, c->stream));
    solve_rows<double>(c->dscr[0], c->dscr[1], nullptr, P<double>(c->tmp[1]), c->Lf,
                       P<double>(c->tmp[0]), P<double>(c->rhs2), c->rownorm, s, R, n, 1.0, c->status,
                       c->L());
  }
  CKS(sync_read(c));
  CK(cudaMemcpy(out, c->dscr[1], cnt * 8, cudaMemcpyDeviceToHost));
  if (c->status_h[0] & 0xffff) {
    CK(cudaMemset(c->status, 0, 16));
    return c->fail(CPALS_E_SINGULAR, "Gamma not finite");
  }
  return CPALS_OK;
}

cpals_status cpals_get_state(cpals_ctx* c, int which, int n, double* out) {
  CKS(ready(c));
  if (n < 0 || n >= c->N || !out || which < 0 || which > 1) return c->fail(CPALS_E_INVALID, "bad argument");
  Join j(c);
  CK(cudaMemcpyAsync(out, which == 0 ? c->Ap[n] : c->dA[n], c->dims[n] * c->R * 8,
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return CPALS_OK;
}

cpals_status cpals_set_profiling(cpals_ctx* c, int enable) {
  if (!c) return CPALS_E_INVALID;
  if ((enable != 0) != c->profiling) drop_graphs(c);
  c->profiling = enable != 0;
  return CPALS_OK;
}

cpals_status cpals_reset_stats(cpals_ctx* c) {
  if (!c) return CPALS_E_INVALID;
  c->launches = 0;
  c->fl_launches = 0;
  c->fl_ms = c->fl_bytes = c->fl_flops = 0;
  c->pc_launches = 0;
  c->pc_ms = c->pc_bytes = 0;
  return CPALS_OK;
}

cpals_status cpals_get_stats(cpals_ctx* c, int kind, int64_t* launches, double* total_ms,
                             double* bytes, double* flops) {
  if (!c) return CPALS_E_INVALID;
  if (kind == 0) {
    if (launches) *launches = c->fl_launches;
    if (total_ms) *total_ms = c->fl_ms;
    if (bytes) *bytes = c->fl_bytes;
    if (flops) *flops = c->fl_flops;
  } else if (kind == 1) {
    if (launches) *launches = c->launches;
    if (total_ms) *total_ms = 0;
    if (bytes) *bytes = 0;
    if (flops) *flops = 0;
  } else if (kind == 2) {
    if (launches) *launches = c->pc_launches;
    if (total_ms) *total_ms = c->pc_ms;
    if (bytes) *bytes = c->pc_bytes;
    if (flops) *flops = 0;
  } else {
    return c->fail(CPALS_E_INVALID, "kind must be 0, 1 or 2");
  }
  return CPALS_OK;
}

cpals_status cpals_set_normal_arith(cpals_ctx* c, int arith) {
  if (!c || (arith != CPALS_NE_FP64 && arith != CPALS_NE_DOUBLE_FLOAT)) return CPALS_E_INVALID;
  if (arith == CPALS_NE_DOUBLE_FLOAT && is64(c))
    return c->fail(CPALS_E_UNSUPPORTED, "double-float normal equations need an FP32 or MIXED_BF16 context");
  CK(cudaStreamSynchronize(c->stream));     // no captured graph still running
  drop_graphs(c);
  c->dfm = arith == CPALS_NE_DOUBLE_FLOAT;
  c->have_factors = false;
  c->ops_built = false;
  return CPALS_OK;
}

cpals_status cpals_set_step_size(cpals_ctx* c, const double* lam) {
  if (!c) return CPALS_E_INVALID;
  double v[kMaxModes];
  for (int n = 0; n < c->N; n++) {
    v[n] = lam ? lam[n] : 1.0;
    if (!(v[n] > 0.0 && v[n] <= 2.0)) return c->fail(CPALS_E_INVALID, "step size outside (0, 2]");
  }
  CK(cudaStreamSynchronize(c->stream));     // no captured graph still running
  drop_graphs(c);                           // the step sizes are kernel arguments
  for (int n = 0; n < c->N; n++) c->lam[n] = v[n];
  return CPALS_OK;
}

cpals_status cpals_set_symmetric(cpals_ctx* c, int m1, int m2) {
  if (!c) return CPALS_E_INVALID;
  const bool clear = m1 < 0 && m2 < 0;
  if (!clear) {
    if (m1 < 0 || m2 <= m1 || m2 >= c->N) return c->fail(CPALS_E_INVALID, "need 0 <= m1 < m2 < N");
    if (c->dims[m1] != c->dims[m2]) return c->fail(CPALS_E_INVALID, "tied modes differ in size");
    if (tied(c, m1)) return c->fail(CPALS_E_INVALID, "m1 is itself tied");
    for (int k = 0; k < c->N; k++)
      if (c->tie[k] == m2) return c->fail(CPALS_E_INVALID, "m2 already has a tied partner");
  }
  CK(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  if (clear)
    for (int k = 0; k < c->N; k++) c->tie[k] = -1;
  else
    c->tie[m2] = m1;
  c->tied_any = false;
  for (int k = 0; k < c->N; k++) c->tied_any = c->tied_any || tied(c, k);
  c->have_factors = false;                  // cpals_init_factors applies the tie
  c->ops_built = false;
  return CPALS_OK;
}

cpals_status cpals_set_wait_limit(cpals_ctx* c, uint64_t cycles) {
  if (!c) return CPALS_E_INVALID;
  c->wait_limit = cycles;
  drop_graphs(c);   // the bound is a launch parameter of the captured kernels
  return CPALS_OK;
}

cpals_status cpals_set_pp_stop_tol(cpals_ctx* c, double tol) {
  if (!c) return CPALS_E_INVALID;
  if (!(tol >= 0.0)) return c->fail(CPALS_E_INVALID, "pp stop tolerance must be >= 0");
  c->pp_stop_tol = tol;
  return CPALS_OK;
}

cpals_status cpals_set_device_loop(cpals_ctx* c, int enable) {
  if (!c) return CPALS_E_INVALID;
  c->device_loop = enable != 0;
  return CPALS_OK;
}

int cpals_device_loop_active(const cpals_ctx* c) {
  return (c && c->device_loop && c->graphs && !c->profiling && c->loop_note.empty()) ? 1 : 0;
}

cpals_status cpals_set_graphs(cpals_ctx* c, int enable) {
  if (!c) return CPALS_E_INVALID;
  if (!enable) drop_graphs(c);
  c->graphs = enable != 0;
  return CPALS_OK;
}

cpals_status cpals_cost_model(const int64_t* dims, int N, int R, int kind, double* flops) {
  if (!dims || !flops || N < 3 || N > kMaxModes || R < 1) return CPALS_E_INVALID;
  for (int i = 0; i < N; i++)
    if (dims[i] < 1) return CPALS_E_INVALID;
  double f = 0;
  const int h = (N + 1) / 2;
  auto chain_cost = [&](std::vector<int> modes, int keep) {
    double cost = 0;
    while (modes.size() > 1) {
      int pos = (int)modes.size() - 1;
      if (modes[pos] == keep) pos--;
      double sz = R;
      for (int m : modes) sz *= (double)dims[m];
      cost += 2.0 * sz;
      modes.erase(modes.begin() + pos);
    }
    return cost;
  };
  double total = 1;
  for (int i = 0; i < N; i++) total *= (double)dims[i];
  if (kind == 0) {
    std::vector<int> Lm, Rm;
    for (int k = 0; k < h; k++) Lm.push_back(k);
    for (int k = h; k < N; k++) Rm.push_back(k);
    f = 2 * 2.0 * total * R;
    for (int n = 0; n < h; n++) f += chain_cost(Lm, n);
    for (int n = h; n < N; n++) f += chain_cost(Rm, n);
  } else if (kind == 1) {
    f = 3 * 2.0 * total * R;
    for (int l = 3; l <= N - 1; l++)
      for (int i = 0; i <= l; i++)
        for (int j = i + 1; j <= l; j++) {
          int pi, pj, w;
          tree_parent(l, i, j, &pi, &pj, &w);
          double sz = R;
          for (int m : level_modes(N, l - 1, pi, pj)) sz *= (double)dims[m];
          f += 2.0 * sz;
        }
  } else if (kind == 2) {
    for (int n = 0; n < N; n++) {
      for (int i = 0; i < N; i++)
        if (i != n) f += 2.0 * dims[i] * dims[n] * R;
      f += 4.0 * dims[n] * R * R;
    }
  } else if (kind == 3) {
    const double s = (double)dims[0];
    for (int l = 2; l <= N - 1; l++) {
      const double comb = (double)(l + 1) * l / 2.0;
      f += comb * std::pow(s, N - l + 2);
    }
    f *= 2.0 * R;
  } else {
    return CPALS_E_INVALID;
  }
  *flops = f;
  return CPALS_OK;
}

}  // extern "C"
