// C ABI of libtaser: argument validation and kernel dispatch (see include/taser.h).
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace taser {
cudaError_t build_T(int kind, int64_t batch, int B, int P, int N, const void* X, const void* y, float* Tt,
                    float* D, uint32_t* flags, cudaStream_t st);
cudaError_t spectral(int64_t batch, int N, const float* Tt, float alpha, int hint, float* tau, float* nrm,
                     cudaStream_t st);
cudaError_t spectral_qpsk(int64_t batch, int U, const float* Tt, int sign, float alpha, float* tau, float* nrm,
                          cudaStream_t st);
cudaError_t unfolded(bool backward, int precision, int64_t batch, int N, const float* Tt, const float* D,
                     const float* inv_norm, const float* alpha_t, int t_max, int c, float* ckpt, float* soft,
                     int8_t* s_hat, const float* grad_soft, float* grad_tau, float* grad_alpha, cudaStream_t st);
size_t unfolded_backward_smem(int N, int c);
size_t unfolded_tc_backward_smem(int c);
size_t uneven_workspace_bytes(int64_t n_items);
cudaError_t detect_uneven(int64_t n_items, const taser_item* items, const float* T_pool, const float* D_pool,
                          const float* tau, int precision, int literal, float* L_pool, int8_t* s_pool,
                          uint32_t* flags, void* workspace, const taser_uneven_tuning* tuning, cudaStream_t st);
cudaError_t detect_fp32(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                        int literal, float* L, int8_t* s, uint32_t* flags, cudaStream_t st);
cudaError_t detect_tc(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                      int literal, bool fp16, float* L, int8_t* s, uint32_t* flags, cudaStream_t st);
cudaError_t detect_fx14(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max, float* L,
                        int8_t* s, uint32_t* flags, cudaStream_t st);
cudaError_t detect_fp32_monitored(int64_t batch, int N, const float* Tt, const float* D, const float* tau,
                                  int t_max, int literal, float ascent_tol, double* obj, float* L, int8_t* s,
                                  uint32_t* flags, cudaStream_t st);
cudaError_t detect_tc_monitored(int64_t batch, int N, const float* Tt, const float* D, const float* tau, int t_max,
                                int literal, bool fp16, float ascent_tol, double* obj, float* L, int8_t* s,
                                uint32_t* flags, cudaStream_t st);
}  // namespace taser

namespace {

thread_local char g_err[512];

taser_status fail(taser_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

taser_status ok() {
  g_err[0] = '\0';
  return TASER_OK;
}

taser_status from_cuda(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return ok();
  return fail(TASER_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// NVTX range over an entry point (host side: argument checks and the enqueue of its
// kernels), so timelines and ncu's --nvtx filters can attribute the kernels to the call.
// Without an attached tool the NVTX calls return at once.
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
  CallRange(const CallRange&) = delete;
  CallRange& operator=(const CallRange&) = delete;
};

#define TASER_REQUIRE(cond, ...)                                  \
  do {                                                            \
    if (!(cond)) return fail(TASER_ERR_INVALID_ARG, __VA_ARGS__); \
  } while (0)

#define TASER_REQUIRE_PTR(p, name)                                                        \
  do {                                                                                    \
    TASER_REQUIRE((p) != nullptr, "%s must not be NULL", name);                           \
    TASER_REQUIRE(aligned16(p), "%s must be 16-byte aligned", name);                      \
  } while (0)

}  // namespace

extern "C" {

int taser_problem_size(int kind, int U_or_K) {
  if (U_or_K <= 0) return -1;
  switch (kind) {
    case TASER_MIMO_BPSK: return U_or_K + 1;
    case TASER_MIMO_QPSK: return 2 * U_or_K + 1;
    case TASER_SIMO_JED_BPSK: return U_or_K;
    case TASER_SIMO_JED_QPSK: return U_or_K >= 2 ? 2 * U_or_K - 1 : -1;
    default: return -1;
  }
}

const char* taser_status_string(int status) {
  switch (status) {
    case TASER_OK: return "ok";
    case TASER_ERR_INVALID_ARG: return "invalid argument";
    case TASER_ERR_UNSUPPORTED: return "unsupported configuration";
    case TASER_ERR_CUDA: return "CUDA error";
    case TASER_ERR_TIMEOUT: return "device wait timed out";
    case TASER_ERR_NUMERIC: return "numeric error";
    default: return "unknown status";
  }
}

const char* taser_last_error(void) { return g_err; }

taser_status taser_build_T(int kind, int64_t batch, int B, int U_or_K, const void* H_or_Y, const void* y,
                           float alpha, float* T_tilde, float* D, float* tau, float* spec_norm, uint32_t* flags,
                           void* stream) {
  const CallRange nvtx_range("taser_build_T");
  TASER_REQUIRE(kind == TASER_MIMO_BPSK || kind == TASER_MIMO_QPSK || kind == TASER_SIMO_JED_BPSK ||
                    kind == TASER_SIMO_JED_QPSK,
                "unknown problem kind %d", kind);
  TASER_REQUIRE(batch >= 0, "batch must be >= 0 (got %lld)", (long long)batch);
  TASER_REQUIRE(B >= 1, "B must be >= 1 (got %d)", B);
  TASER_REQUIRE(alpha > 0.f && alpha < 1.f, "alpha must lie in (0, 1) (got %g)", (double)alpha);
  const bool jed = kind == TASER_SIMO_JED_BPSK || kind == TASER_SIMO_JED_QPSK;
  if (jed) {
    TASER_REQUIRE(U_or_K >= 2 && U_or_K <= 33, "JED needs 2 <= K <= 33 (got %d)", U_or_K);
    TASER_REQUIRE(y == nullptr, "y must be NULL for JED");
  } else {
    TASER_REQUIRE(U_or_K >= 1 && U_or_K <= 32, "MIMO needs 1 <= U <= 32 (got %d)", U_or_K);
  }
  const int N = taser_problem_size(kind, U_or_K);
  TASER_REQUIRE(N >= 2 && N <= TASER_MAX_N, "problem size N = %d outside [2, %d]", N, TASER_MAX_N);
  if (batch == 0) return ok();
  TASER_REQUIRE_PTR(H_or_Y, "H_or_Y");
  if (!jed) TASER_REQUIRE_PTR(y, "y");
  TASER_REQUIRE_PTR(T_tilde, "T_tilde");
  TASER_REQUIRE_PTR(D, "D");
  if (tau != nullptr) TASER_REQUIRE(aligned16(tau), "tau must be 16-byte aligned");
  if (spec_norm != nullptr) TASER_REQUIRE(aligned16(spec_norm), "spec_norm must be 16-byte aligned");
  if (flags != nullptr) TASER_REQUIRE(aligned16(flags), "flags must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int P = jed ? U_or_K - 1 : U_or_K;
  cudaError_t e = taser::build_T(kind, batch, B, P, N, H_or_Y, y, T_tilde, D, flags, st);
  if (e == cudaErrorNotSupported) return fail(TASER_ERR_UNSUPPORTED, "no build kernel for %d columns", P + 1);
  if (e != cudaSuccess) return from_cuda(e, "build_T");
  if (tau == nullptr) return ok();
  return taser_step_size(batch, N, T_tilde, kind, alpha, tau, spec_norm, stream);
}

taser_status taser_step_size(int64_t batch, int N, const float* T_tilde, int structure, float alpha, float* tau,
                             float* spec_norm, void* stream) {
  const CallRange nvtx_range("taser_step_size");
  TASER_REQUIRE(batch >= 0, "batch must be >= 0 (got %lld)", (long long)batch);
  TASER_REQUIRE(N >= 2 && N <= TASER_MAX_N, "N = %d outside [2, %d]", N, TASER_MAX_N);
  TASER_REQUIRE(alpha > 0.f && alpha < 1.f, "alpha must lie in (0, 1) (got %g)", (double)alpha);
  TASER_REQUIRE(structure == TASER_GENERIC_SYMMETRIC || structure == TASER_MIMO_BPSK ||
                    structure == TASER_MIMO_QPSK || structure == TASER_SIMO_JED_BPSK ||
                    structure == TASER_SIMO_JED_QPSK,
                "unknown structure %d", structure);
  TASER_REQUIRE((structure != TASER_MIMO_QPSK && structure != TASER_SIMO_JED_QPSK) || N % 2 == 1,
                "QPSK structure needs odd N (got %d)", N);
  if (batch == 0) return ok();
  TASER_REQUIRE_PTR(T_tilde, "T_tilde");
  TASER_REQUIRE_PTR(tau, "tau");
  if (spec_norm != nullptr) TASER_REQUIRE(aligned16(spec_norm), "spec_norm must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (structure == TASER_MIMO_QPSK || structure == TASER_SIMO_JED_QPSK) {
    // ||T~||_2 equals the norm of its (U+1) x (U+1) complex Hermitian form.
    const int sign = structure == TASER_MIMO_QPSK ? 1 : -1;
    return from_cuda(taser::spectral_qpsk(batch, (N - 1) / 2, T_tilde, sign, alpha, tau, spec_norm, st),
                     "spectral_qpsk");
  }
  // T = A^T A is positive semidefinite (MIMO), T = -A^T A negative semidefinite (JED).
  const int hint = structure == TASER_MIMO_BPSK ? 1 : (structure == TASER_SIMO_JED_BPSK ? -1 : 0);
  return from_cuda(taser::spectral(batch, N, T_tilde, alpha, hint, tau, spec_norm, st), "spectral");
}

taser_status taser_detect(int64_t batch, int N, const float* T_tilde, const float* D, const float* tau, int t_max,
                          int precision, int lnn_mode, float* L, int8_t* s_hat, uint32_t* flags, void* stream) {
  const CallRange nvtx_range("taser_detect");
  TASER_REQUIRE(batch >= 0, "batch must be >= 0 (got %lld)", (long long)batch);
  TASER_REQUIRE(N >= 2 && N <= TASER_MAX_N, "N = %d outside [2, %d]", N, TASER_MAX_N);
  TASER_REQUIRE(t_max >= 1, "t_max must be >= 1 (got %d)", t_max);
  TASER_REQUIRE(precision == TASER_FP32 || precision == TASER_BF16_TC || precision == TASER_FP16_TC ||
                    precision == TASER_FIXED14,
                "unknown precision %d", precision);
  TASER_REQUIRE(lnn_mode == TASER_LNN_FIXED || lnn_mode == TASER_LNN_LITERAL, "unknown lnn_mode %d", lnn_mode);
  if (precision == TASER_FIXED14 && lnn_mode != TASER_LNN_FIXED)
    return fail(TASER_ERR_UNSUPPORTED, "TASER_FIXED14 keeps L~_NN constant: only TASER_LNN_FIXED is available");
  if (batch == 0) return ok();
  TASER_REQUIRE_PTR(T_tilde, "T_tilde");
  TASER_REQUIRE_PTR(D, "D");
  TASER_REQUIRE_PTR(tau, "tau");
  TASER_REQUIRE_PTR(s_hat, "s_hat");
  if (L != nullptr) TASER_REQUIRE(aligned16(L), "L must be 16-byte aligned");
  if (flags != nullptr) TASER_REQUIRE(aligned16(flags), "flags must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int literal = lnn_mode == TASER_LNN_LITERAL;
  if (precision == TASER_FIXED14) {
    return from_cuda(taser::detect_fx14(batch, N, T_tilde, D, tau, t_max, L, s_hat, flags, st), "detect_fx14");
  }
  if (precision != TASER_FP32 && taser::bucket_of(N) >= 16) {
    return from_cuda(taser::detect_tc(batch, N, T_tilde, D, tau, t_max, literal, precision == TASER_FP16_TC, L,
                                      s_hat, flags, st),
                     "detect_tc");
  }
  return from_cuda(taser::detect_fp32(batch, N, T_tilde, D, tau, t_max, literal, L, s_hat, flags, st),
                   "detect_fp32");
}

taser_status taser_detect_monitored(int64_t batch, int N, const float* T_tilde, const float* D, const float* tau,
                                    int t_max, int precision, int lnn_mode, float ascent_tol, double* objective,
                                    float* L, int8_t* s_hat, uint32_t* flags, void* stream) {
  const CallRange nvtx_range("taser_detect_monitored");
  TASER_REQUIRE(batch >= 0, "batch must be >= 0 (got %lld)", (long long)batch);
  TASER_REQUIRE(N >= 2 && N <= TASER_MAX_N, "N = %d outside [2, %d]", N, TASER_MAX_N);
  TASER_REQUIRE(t_max >= 1, "t_max must be >= 1 (got %d)", t_max);
  TASER_REQUIRE(precision == TASER_FP32 || precision == TASER_BF16_TC || precision == TASER_FP16_TC ||
                    precision == TASER_FIXED14,
                "unknown precision %d", precision);
  TASER_REQUIRE(lnn_mode == TASER_LNN_FIXED || lnn_mode == TASER_LNN_LITERAL, "unknown lnn_mode %d", lnn_mode);
  TASER_REQUIRE(ascent_tol >= 0.f, "ascent_tol must be >= 0 (got %g)", (double)ascent_tol);
  if (precision == TASER_FIXED14)
    return fail(TASER_ERR_UNSUPPORTED, "objective monitoring is not available for TASER_FIXED14");
  const bool tc = precision != TASER_FP32 && taser::bucket_of(N) >= 16;
  if (tc && taser::bucket_of(N) > 32)
    return fail(TASER_ERR_UNSUPPORTED, "objective monitoring on the tensor cores needs N <= 33 (got %d)", N);
  if (batch == 0) return ok();
  TASER_REQUIRE_PTR(T_tilde, "T_tilde");
  TASER_REQUIRE_PTR(D, "D");
  TASER_REQUIRE_PTR(tau, "tau");
  TASER_REQUIRE_PTR(s_hat, "s_hat");
  if (L != nullptr) TASER_REQUIRE(aligned16(L), "L must be 16-byte aligned");
  if (flags != nullptr) TASER_REQUIRE(aligned16(flags), "flags must be 16-byte aligned");
  if (objective != nullptr) TASER_REQUIRE(aligned16(objective), "objective must be 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int literal = lnn_mode == TASER_LNN_LITERAL;
  if (tc) {
    return from_cuda(taser::detect_tc_monitored(batch, N, T_tilde, D, tau, t_max, literal,
                                                precision == TASER_FP16_TC, ascent_tol, objective, L, s_hat, flags,
                                                st),
                     "detect_tc_monitored");
  }
  return from_cuda(taser::detect_fp32_monitored(batch, N, T_tilde, D, tau, t_max, literal, ascent_tol, objective, L,
                                                s_hat, flags, st),
                   "detect_fp32_monitored");
}

}  // extern "C"

namespace {
// Side stream (per host thread and device) that carries taser_run_host's host-to-device
// copies, so chunk k + 1 is in flight while chunk k is detected on the caller's stream.
// Created on first use and kept for the thread's lifetime.
struct CopyLane {
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, copied = nullptr;
};
cudaError_t copy_lane(CopyLane*& out) {
  thread_local CopyLane lanes[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  CopyLane& c = lanes[dev];
  if (c.stream == nullptr) {
    e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.copied, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      c = CopyLane{};
      return e;
    }
  }
  out = &c;
  return cudaSuccess;
}

// Instances per pipelined chunk of taser_run_host: large enough that every kernel still
// fills the GPU, small enough that the copy of the first chunk is a small part of the whole.
constexpr int64_t kHostChunk = 8192;

struct HostLayout {
  size_t x, y, t, d, tau, s, flags, total;
};
size_t up256(size_t v) { return (v + 255) & ~size_t(255); }
bool host_layout(int kind, int64_t batch, int B, int M, HostLayout& L) {
  const int N = taser_problem_size(kind, M);
  if (N < 2 || batch < 0 || B < 1) return false;
  const bool jed = kind == TASER_SIMO_JED_BPSK || kind == TASER_SIMO_JED_QPSK;
  size_t off = 0;
  L.x = off; off = up256(off + size_t(batch) * B * M * 8);
  L.y = off; off = up256(off + (jed ? 0 : size_t(batch) * B * 8));
  L.t = off; off = up256(off + size_t(batch) * N * N * 4);
  L.d = off; off = up256(off + size_t(batch) * N * 4);
  L.tau = off; off = up256(off + size_t(batch) * 4);
  L.s = off; off = up256(off + size_t(batch) * (N - 1));
  L.flags = off; off = up256(off + size_t(batch) * 4);
  L.total = off;
  return true;
}
}  // namespace

extern "C" {

size_t taser_host_workspace_bytes(int kind, int64_t batch, int B, int U_or_K) {
  HostLayout L;
  if (!host_layout(kind, batch, B, U_or_K, L)) return 0;
  return L.total;
}

taser_status taser_run_host(int kind, int64_t batch, int B, int U_or_K, const void* H_or_Y, const void* y,
                            float alpha, int t_max, int precision, int lnn_mode, void* workspace,
                            size_t workspace_bytes, int8_t* s_hat, uint32_t* flags, void* stream) {
  const CallRange nvtx_range("taser_run_host");
  TASER_REQUIRE(kind == TASER_MIMO_BPSK || kind == TASER_MIMO_QPSK || kind == TASER_SIMO_JED_BPSK ||
                    kind == TASER_SIMO_JED_QPSK,
                "unknown problem kind %d", kind);
  TASER_REQUIRE(batch >= 0, "batch must be >= 0 (got %lld)", (long long)batch);
  TASER_REQUIRE(t_max >= 1, "t_max must be >= 1 (got %d)", t_max);
  HostLayout L;
  TASER_REQUIRE(host_layout(kind, batch, B, U_or_K, L), "invalid problem shape");
  if (batch == 0) return ok();
  const bool jed = kind == TASER_SIMO_JED_BPSK || kind == TASER_SIMO_JED_QPSK;
  TASER_REQUIRE(H_or_Y != nullptr, "H_or_Y must not be NULL");
  TASER_REQUIRE(jed || y != nullptr, "y must not be NULL");
  TASER_REQUIRE(s_hat != nullptr, "s_hat must not be NULL");
  TASER_REQUIRE(workspace != nullptr && (reinterpret_cast<uintptr_t>(workspace) & 255u) == 0,
                "workspace must be a 256-byte aligned device pointer");
  TASER_REQUIRE(workspace_bytes >= L.total, "workspace too small: %zu < %zu bytes", workspace_bytes, L.total);
  const int N = taser_problem_size(kind, U_or_K);
  char* w = static_cast<char*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CopyLane* lane = nullptr;
  cudaError_t e = copy_lane(lane);
  if (e != cudaSuccess) return from_cuda(e, "copy stream");
  // The copies may only start once earlier work on `stream` (which may still read the
  // workspace) is done: fork the side stream from it.
  e = cudaEventRecord(lane->fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(lane->stream, lane->fork, 0);
  if (e != cudaSuccess) return from_cuda(e, "fork copy stream");
  const size_t xrow = size_t(B) * U_or_K * 8, yrow = size_t(B) * 8;
  float* Tt = reinterpret_cast<float*>(w + L.t);
  float* D = reinterpret_cast<float*>(w + L.d);
  float* tau = reinterpret_cast<float*>(w + L.tau);
  int8_t* s = reinterpret_cast<int8_t*>(w + L.s);
  uint32_t* fl = reinterpret_cast<uint32_t*>(w + L.flags);
  for (int64_t c0 = 0; c0 < batch; c0 += kHostChunk) {
    const int64_t nc = batch - c0 < kHostChunk ? batch - c0 : kHostChunk;
    char* xk = w + L.x + size_t(c0) * xrow;
    char* yk = w + L.y + size_t(c0) * yrow;
    e = cudaMemcpyAsync(xk, static_cast<const char*>(H_or_Y) + size_t(c0) * xrow, size_t(nc) * xrow,
                        cudaMemcpyHostToDevice, lane->stream);
    if (e != cudaSuccess) return from_cuda(e, "copy H_or_Y");
    if (!jed) {
      e = cudaMemcpyAsync(yk, static_cast<const char*>(y) + size_t(c0) * yrow, size_t(nc) * yrow,
                          cudaMemcpyHostToDevice, lane->stream);
      if (e != cudaSuccess) return from_cuda(e, "copy y");
    }
    // The event is re-recorded per chunk: each wait binds to the record just before it.
    e = cudaEventRecord(lane->copied, lane->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, lane->copied, 0);
    if (e != cudaSuccess) return from_cuda(e, "join copy stream");
    float* Tk = Tt + size_t(c0) * N * N;
    float* Dk = D + size_t(c0) * N;
    int8_t* sk = s + size_t(c0) * (N - 1);
    taser_status rs = taser_build_T(kind, nc, B, U_or_K, xk, jed ? nullptr : yk, alpha, Tk, Dk, tau + c0,
                                    nullptr, fl + c0, stream);
    if (rs != TASER_OK) return rs;
    rs = taser_detect(nc, N, Tk, Dk, tau + c0, t_max, precision, lnn_mode, nullptr, sk, fl + c0, stream);
    if (rs != TASER_OK) return rs;
    e = cudaMemcpyAsync(s_hat + size_t(c0) * (N - 1), sk, size_t(nc) * (N - 1), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return from_cuda(e, "copy s_hat");
    if (flags != nullptr) {
      e = cudaMemcpyAsync(flags + c0, fl + c0, size_t(nc) * 4, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return from_cuda(e, "copy flags");
    }
  }
  return ok();
}

}  // extern "C"

namespace taser {
// Records `msg` as the thread's last error (taser_last_error) and returns `st`.
taser_status report(taser_status st, const char* msg) { return fail(st, "%s", msg); }
}  // namespace taser

extern "C" {

namespace {
bool unfolded_tc_path(int precision, int N) {
  return (precision == TASER_BF16_TC || precision == TASER_FP16_TC) && taser::bucket_of(N) == 32;
}
}  // namespace

taser_status taser_unfolded_forward(int64_t batch, int N, const float* T_tilde, const float* D, const float* inv_norm,
                                    const float* alpha_t, int t_max, int c, int precision, float* ckpt, float* soft,
                                    int8_t* s_hat, void* stream) {
  const CallRange nvtx_range("taser_unfolded_forward");
  TASER_REQUIRE(batch >= 0, "batch must be >= 0 (got %lld)", (long long)batch);
  TASER_REQUIRE(N >= 2 && N <= 33, "unfolded TASER supports 2 <= N <= 33 (got %d)", N);
  TASER_REQUIRE(t_max >= 1, "t_max must be >= 1 (got %d)", t_max);
  TASER_REQUIRE(c >= 1 && c <= t_max, "checkpoint spacing c must lie in [1, t_max] (got %d)", c);
  TASER_REQUIRE(precision == TASER_FP32 || precision == TASER_BF16_TC || precision == TASER_FP16_TC ||
                    precision == TASER_FIXED14,
                "unknown precision %d", precision);
  if (precision == TASER_FIXED14) return fail(TASER_ERR_UNSUPPORTED, "unfolded TASER has no fixed-point datapath");
  if (batch == 0) return ok();
  TASER_REQUIRE_PTR(T_tilde, "T_tilde");
  TASER_REQUIRE_PTR(D, "D");
  TASER_REQUIRE_PTR(inv_norm, "inv_norm");
  TASER_REQUIRE_PTR(alpha_t, "alpha_t");
  TASER_REQUIRE_PTR(soft, "soft");
  if (ckpt != nullptr) TASER_REQUIRE(aligned16(ckpt), "ckpt must be 16-byte aligned");
  if (s_hat != nullptr) TASER_REQUIRE(aligned16(s_hat), "s_hat must be 16-byte aligned");
  return from_cuda(taser::unfolded(false, precision, batch, N, T_tilde, D, inv_norm, alpha_t, t_max, c, ckpt, soft,
                                   s_hat, nullptr, nullptr, nullptr, static_cast<cudaStream_t>(stream)),
                   "unfolded_forward");
}

taser_status taser_unfolded_backward(int64_t batch, int N, const float* T_tilde, const float* D,
                                     const float* inv_norm, const float* alpha_t, int t_max, int c, int precision,
                                     const float* ckpt, const float* grad_soft, float* grad_tau, float* grad_alpha,
                                     void* stream) {
  const CallRange nvtx_range("taser_unfolded_backward");
  TASER_REQUIRE(batch >= 0, "batch must be >= 0 (got %lld)", (long long)batch);
  TASER_REQUIRE(N >= 2 && N <= 33, "unfolded TASER supports 2 <= N <= 33 (got %d)", N);
  TASER_REQUIRE(t_max >= 1, "t_max must be >= 1 (got %d)", t_max);
  TASER_REQUIRE(c >= 1 && c <= t_max, "checkpoint spacing c must lie in [1, t_max] (got %d)", c);
  TASER_REQUIRE(precision == TASER_FP32 || precision == TASER_BF16_TC || precision == TASER_FP16_TC ||
                    precision == TASER_FIXED14,
                "unknown precision %d", precision);
  if (precision == TASER_FIXED14) return fail(TASER_ERR_UNSUPPORTED, "unfolded TASER has no fixed-point datapath");
  {
    const size_t need = unfolded_tc_path(precision, N) ? taser::unfolded_tc_backward_smem(c)
                                                       : taser::unfolded_backward_smem(N, c);
    TASER_REQUIRE(need <= 227 * 1024,
                  "checkpoint spacing c = %d needs %zu bytes of shared memory per block (limit 232448)", c, need);
  }
  if (batch == 0) return ok();
  TASER_REQUIRE_PTR(T_tilde, "T_tilde");
  TASER_REQUIRE_PTR(D, "D");
  TASER_REQUIRE_PTR(inv_norm, "inv_norm");
  TASER_REQUIRE_PTR(alpha_t, "alpha_t");
  TASER_REQUIRE_PTR(ckpt, "ckpt");
  TASER_REQUIRE_PTR(grad_soft, "grad_soft");
  TASER_REQUIRE_PTR(grad_tau, "grad_tau");
  if (grad_alpha != nullptr) TASER_REQUIRE(aligned16(grad_alpha), "grad_alpha must be 16-byte aligned");
  return from_cuda(taser::unfolded(true, precision, batch, N, T_tilde, D, inv_norm, alpha_t, t_max, c,
                                   const_cast<float*>(ckpt), nullptr, nullptr, grad_soft, grad_tau, grad_alpha,
                                   static_cast<cudaStream_t>(stream)),
                   "unfolded_backward");
}

}  // extern "C"

extern "C" {

size_t taser_uneven_workspace_bytes(int64_t n_items) {
  if (n_items < 0 || n_items > 0x7fffffff) return 0;
  return taser::uneven_workspace_bytes(n_items);
}

taser_status taser_detect_uneven(int64_t n_items, const taser_item* items, const float* T_pool, const float* D_pool,
                                 const float* tau, int precision, int lnn_mode, float* L_pool, int8_t* s_pool,
                                 uint32_t* flags, void* workspace, size_t workspace_bytes,
                                 const taser_uneven_tuning* tuning, void* stream) {
  const CallRange nvtx_range("taser_detect_uneven");
  TASER_REQUIRE(n_items >= 0 && n_items <= 0x7fffffff, "n_items must lie in [0, 2^31) (got %lld)",
                (long long)n_items);
  TASER_REQUIRE(precision == TASER_FP32 || precision == TASER_BF16_TC || precision == TASER_FP16_TC ||
                    precision == TASER_FIXED14,
                "unknown precision %d", precision);
  TASER_REQUIRE(lnn_mode == TASER_LNN_FIXED || lnn_mode == TASER_LNN_LITERAL, "unknown lnn_mode %d", lnn_mode);
  if (precision == TASER_FIXED14 && lnn_mode != TASER_LNN_FIXED)
    return fail(TASER_ERR_UNSUPPORTED, "TASER_FIXED14 keeps L~_NN constant: only TASER_LNN_FIXED is available");
  if (n_items == 0) return ok();
  TASER_REQUIRE(items != nullptr && (reinterpret_cast<uintptr_t>(items) & 7u) == 0, "items must be 8-byte aligned");
  TASER_REQUIRE(T_pool != nullptr && D_pool != nullptr && tau != nullptr && s_pool != nullptr,
                "T_pool, D_pool, tau and s_pool must not be NULL");
  TASER_REQUIRE(workspace != nullptr && (reinterpret_cast<uintptr_t>(workspace) & 255u) == 0,
                "workspace must be a 256-byte aligned device pointer");
  TASER_REQUIRE(workspace_bytes >= taser::uneven_workspace_bytes(n_items), "workspace too small: %zu < %zu bytes",
                workspace_bytes, taser::uneven_workspace_bytes(n_items));
  if (tuning != nullptr) {
    for (int b = 0; b < 4; ++b)
      TASER_REQUIRE(tuning->blocks_per_sm[b] >= 0 && tuning->pop[b] >= 0 && tuning->pop[b] <= 64,
                    "tuning entry %d out of range", b);
  }
  return from_cuda(taser::detect_uneven(n_items, items, T_pool, D_pool, tau, precision, lnn_mode == TASER_LNN_LITERAL,
                                        L_pool, s_pool, flags, workspace, tuning, static_cast<cudaStream_t>(stream)),
                   "detect_uneven");
}

}  // extern "C"

#ifdef TASER_DEBUG
namespace taser {
namespace dbg {
// Counter collectors of the translation units that hold kernels (TASER_DEBUG_COLLECTOR).
cudaError_t take_build_T(unsigned long long* out);
cudaError_t take_spectral(unsigned long long* out);
cudaError_t take_detect_fp32(unsigned long long* out);
cudaError_t take_detect_tc(unsigned long long* out);
cudaError_t take_detect_fx14(unsigned long long* out);
cudaError_t take_unfolded(unsigned long long* out);
cudaError_t take_unfolded_tc(unsigned long long* out);
cudaError_t take_uneven(unsigned long long* out);
}  // namespace dbg
cudaError_t debug_drop_copy(int64_t inst, int chunk);
}  // namespace taser
#endif

extern "C" {

taser_status taser_debug_report(uint64_t* fails, uint64_t* first, uint64_t* nonfinite) {
  TASER_REQUIRE(fails != nullptr && first != nullptr && nonfinite != nullptr,
                "fails, first and nonfinite must not be NULL");
#ifdef TASER_DEBUG
  using namespace taser::dbg;
  cudaError_t (*const takes[])(unsigned long long*) = {take_build_T,     take_spectral, take_detect_fp32,
                                                        take_detect_tc,   take_detect_fx14,
                                                        take_unfolded,    take_unfolded_tc, take_uneven};
  unsigned long long acc[3] = {0ull, 0ull, 0ull};
  for (auto take : takes) {
    const cudaError_t e = take(acc);
    if (e != cudaSuccess) return from_cuda(e, "debug counters");
  }
  *fails = acc[0];
  *first = acc[1];
  *nonfinite = acc[2];
  return ok();
#else
  return fail(TASER_ERR_UNSUPPORTED, "release build: the debug counters exist in libtaser_debug.so only");
#endif
}

taser_status taser_debug_drop_copy(int64_t instance, int chunk) {
#ifdef TASER_DEBUG
  return from_cuda(taser::debug_drop_copy(instance < 0 ? -1 : instance, instance < 0 ? -1 : chunk),
                   "debug_drop_copy");
#else
  (void)instance;
  (void)chunk;
  return fail(TASER_ERR_UNSUPPORTED, "release build: fault injection exists in libtaser_debug.so only");
#endif
}

}  // extern "C"
