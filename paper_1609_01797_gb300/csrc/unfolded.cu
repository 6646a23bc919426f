// Unfolded TASER: Algorithm 1 with a learnable step per iteration, tau_t = alpha_t /
// ||T~||_2, its FP32 forward with checkpoints, and the hand-written adjoint.
//
// Forward (mode "fixed", L~_NN = D_NN):  V_t = L~(t-1) - tau_t tril(2 L~(t-1) T~),
// L~(t) = prox(V_t); soft output x_k = L~(t_max)_{N,k} / D_k (the last row of the
// unit-column factor L = L~ D^-1).  L~(kc) is saved every c iterations.
//
// Adjoint of one step, given Lbar = dloss/dL~(t):
//   G = tril(2 L~(t-1) T~),  u_k = V_{.k} / ||V_{.k}||,
//   Vbar_{.k} = (D_k / ||V_{.k}||) (Lbar_{.k} - u_k (u_k . Lbar_{.k}))  for k < N-1, Vbar_{.N} = 0,
//   taubar_t = - sum_{i >= j} Vbar_ij G_ij,
//   dloss/dL~(t-1) = tril(Vbar - tau_t Vbar (2 T~)).
// Each segment of c iterations is recomputed from its checkpoint and kept in shared
// memory while it is differentiated in reverse.
//
// Mapping as in the FP32 detector: one warp per instance, lane j owns column j of L~, V,
// G, Vbar and Lbar; the column j of T~ stays in registers; rows of L~ and Vbar are
// broadcast from shared memory, so both products keep the triangular skip.  Shared memory
// holds only the lower triangle: row i takes i + 1 floats rounded up to a multiple of 4
// (16-byte rows for the float4 broadcasts), 612 floats at bucket 32 instead of 33 x 36.
#include "common.cuh"

namespace taser {

// Offset (floats) of row i of a packed lower-triangular matrix whose row r holds
// (r + 1) rounded up to 4 floats: with i = 4q + m, 16 q (q + 1) / 2 + 4 m (q + 1).
__host__ __device__ constexpr int tri_off(int i) { return 4 * ((i >> 2) + 1) * (2 * (i >> 2) + (i & 3)); }

template <int NB>
struct UfCfg {
  static constexpr int MAT = tri_off(NB + 1);       // one bucket matrix in smem (rows 0..NB)
  static constexpr int WARPS = 4;                   // forward: warps per block
  // Adjoint: one warp per block, so a block needs only its own (c + 2) packed iterates and
  // c can reach 92 at N = 33; 12 blocks per SM (3 warps per scheduler) at 168 registers.
  static constexpr int BWD_WARPS = 1;
  static constexpr int BWD_MIN_BLOCKS = 12;
};


// 4-byte asynchronous global -> shared copy (completed by cp.async.wait_all).
__device__ __forceinline__ void uf_cp_async4(float* smem_dst, const float* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}

// Column j of T~ as pairs (T~_kj, T~_k+1,j), zero past k = NB.
template <int NB>
struct TPairs {
  static constexpr int P = NB / 2 + 2;
  uint64_t v[P];
};

// acc_i = sum_{k <= i} R[i][k] t[k] for the rows i of a lower-triangular smem matrix R whose
// row padding is zero: one LDS.128 feeds two packed FMAs (even and odd k), and the last
// float4 of a row needs no mask.
template <int NB>
__device__ __forceinline__ float tri_row(const float* R, int i, const TPairs<NB>& t) {
  uint64_t acc = 0ull;
  const float* row = R + tri_off(i);
#pragma unroll
  for (int k4 = 0; k4 <= NB; k4 += 4) {
    if (k4 > i) break;
    const float4 q = *reinterpret_cast<const float4*>(row + k4);
    acc = f2fma(f2pack(q.x, q.y), t.v[k4 / 2], acc);
    if (k4 + 2 <= i) acc = f2fma(f2pack(q.z, q.w), t.v[k4 / 2 + 1], acc);
  }
  float a0, a1;
  f2unpack(acc, a0, a1);
  return a0 + a1;
}

// One forward step on the smem iterate Lin -> Lout (column j of the result also
// returned in l[]).  Returns nothing; l holds L~(t) column j on exit.
template <int NB>
__device__ __forceinline__ void forward_step(const float* Lin, float* Lout, float (&l)[NB + 1],
                                             const TPairs<NB>& tcol, float tau, float Dj, int j) {
  float v[NB + 1];
#pragma unroll
  for (int i = 0; i <= NB; ++i) {
    const float g = 2.f * tri_row<NB>(Lin, i, tcol);
    v[i] = (i >= j) ? fmaf(-tau, g, Lin[tri_off(i) + j]) : 0.f;
  }
  float n2 = 0.f;
#pragma unroll
  for (int i = 0; i <= NB; ++i) n2 = fmaf(v[i], v[i], n2);
  const float sc = n2 > 0.f ? Dj * rsqrtf(n2) : 0.f;
#pragma unroll
  for (int i = 0; i <= NB; ++i) {
    l[i] = v[i] * sc;
    if (i >= j) Lout[tri_off(i) + j] = l[i];
  }
}

template <int NB>
__device__ __forceinline__ void load_tcol(TPairs<NB>& tcol, const float* T, int N, int jr) {
#pragma unroll
  for (int p = 0; p < TPairs<NB>::P; ++p) {
    float v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * p + h;
      const int kr = k <= NB ? bucket_to_real(k, N, NB) : -1;
      v[h] = (jr >= 0 && kr >= 0 && TASER_IN(kr * N + jr, N * N)) ? T[(int64_t)kr * N + jr] : 0.f;
    }
    tcol.v[p] = f2pack(v[0], v[1]);
  }
}

template <int NB>
__device__ __forceinline__ void init_diag(float* L, int j, float Dj, float DN, int lane) {
  for (int idx = lane; idx < UfCfg<NB>::MAT; idx += 32) L[idx] = 0.f;
  __syncwarp();
  if (j < NB) L[tri_off(j) + j] = Dj;
  if (lane == 0) L[tri_off(NB) + NB] = DN;
  __syncwarp();
}

template <int NB>
__global__ void __launch_bounds__(128, 5)
unfolded_forward_kernel(int64_t batch, int N, const float* __restrict__ Tt, const float* __restrict__ Dg,
                        const float* __restrict__ inv_norm, const float* __restrict__ alpha_t, int t_max, int c,
                        float* __restrict__ ckpt, float* __restrict__ soft, int8_t* __restrict__ s_hat) {
  using C = UfCfg<NB>;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t inst = (int64_t)blockIdx.x * C::WARPS + warp;
  if (inst >= batch) return;
  float* buf0 = smem + warp * 2 * C::MAT;
  float* buf1 = buf0 + C::MAT;
  const int j = lane;                                  // lanes >= NB carry zero columns
  const int jr = j < N - 1 ? j : -1;
  const float* T = Tt + inst * (int64_t)N * N;
  TPairs<NB> tcol;
  load_tcol<NB>(tcol, T, N, jr);
  const float Dj = jr >= 0 && TASER_IN(inst * N + jr, batch * N) ? Dg[inst * N + jr] : 0.f;
  const float DN = Dg[inst * N + N - 1];
  const float inv = inv_norm[inst];
  const int n_ckpt = (t_max + c - 1) / c;
  init_diag<NB>(buf0, j < NB ? j : NB, j < NB ? Dj : 0.f, DN, lane);
  float l[NB + 1];
#pragma unroll
  for (int i = 0; i <= NB; ++i) l[i] = (i == j) ? Dj : 0.f;
  float* cur = buf0;
  float* nxt = buf1;
  for (int idx = lane; idx < C::MAT; idx += 32) nxt[idx] = cur[idx];  // keeps L~_NN in both buffers
  __syncwarp();
  for (int t = 0; t < t_max; ++t) {
    if (t % c == 0 && ckpt != nullptr) {
      // checkpoint L~(t) in real indices, full N x N with zeros above the diagonal
      float* out = ckpt + (inst * n_ckpt + t / c) * (int64_t)N * N;
      const int dq = 32 / N, dm = 32 % N;
      int r = lane / N, cc = lane % N;                 // (r, cc) of element e, advanced by 32
      for (int e = lane; e < N * N; e += 32) {
        const int br = r == N - 1 ? NB : r, bc = cc == N - 1 ? NB : cc;
        if (TASER_IN((inst * n_ckpt + t / c) * N * N + e, batch * n_ckpt * N * N) &&
            TASER_IN(tri_off(br) + (bc <= br ? bc : 0), C::MAT))
          out[e] = bc <= br ? cur[tri_off(br) + bc] : 0.f;
        r += dq;
        cc += dm;
        if (cc >= N) { cc -= N; ++r; }
      }
    }
    const float tau = TASER_IN(t, t_max) ? alpha_t[t] * inv : 0.f;
    if (j < NB) forward_step<NB>(cur, nxt, l, tcol, tau, Dj, j);
    __syncwarp();
    float* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  if (jr >= 0 && TASER_IN(inst * (N - 1) + jr, batch * (N - 1))) {
    soft[inst * (N - 1) + jr] = Dj > 0.f ? l[NB] / Dj : 0.f;
    TASER_FINITE(soft[inst * (N - 1) + jr]);
    if (s_hat != nullptr) s_hat[inst * (N - 1) + jr] = l[NB] >= 0.f ? int8_t(1) : int8_t(-1);
  }
}

template <int NB>
__global__ void __launch_bounds__(32 * UfCfg<NB>::BWD_WARPS, UfCfg<NB>::BWD_MIN_BLOCKS)
unfolded_backward_kernel(int64_t batch, int N, const float* __restrict__ Tt, const float* __restrict__ Dg,
                         const float* __restrict__ inv_norm, const float* __restrict__ alpha_t, int t_max, int c,
                         const float* __restrict__ ckpt, const float* __restrict__ grad_soft,
                         float* __restrict__ grad_tau) {
  using C = UfCfg<NB>;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t inst = (int64_t)blockIdx.x * C::BWD_WARPS + warp;
  if (inst >= batch) return;
  // per warp: c + 1 iterates of the segment and the Vbar rows
  float* seg = smem + (int64_t)warp * (c + 2) * C::MAT;
  float* vb = seg + (c + 1) * C::MAT;
  const int j = lane;
  const int jr = j < N - 1 ? j : -1;
  const float* T = Tt + inst * (int64_t)N * N;
  TPairs<NB> tcol;
  load_tcol<NB>(tcol, T, N, jr);
  const float Dj = jr >= 0 && TASER_IN(inst * N + jr, batch * N) ? Dg[inst * N + jr] : 0.f;
  const float inv = inv_norm[inst];
  // The rows of Vbar are written on and below the diagonal only: zero the padding once.
  for (int idx = lane; idx < C::MAT; idx += 32) vb[idx] = 0.f;
  __syncwarp();
  const int n_ckpt = (t_max + c - 1) / c;
  // Lbar(t_max): only the last row, dloss/dL~_{N,k} = dloss/dx_k / D_k
  float lbar[NB + 1];
#pragma unroll
  for (int i = 0; i <= NB; ++i) lbar[i] = 0.f;
  if (jr >= 0 && Dj > 0.f && TASER_IN(inst * (N - 1) + jr, batch * (N - 1)))
    lbar[NB] = grad_soft[inst * (N - 1) + jr] / Dj;

  for (int kc = n_ckpt - 1; kc >= 0; --kc) {
    const int t0 = kc * c, t1 = min(t0 + c, t_max);
    // L~(t0) from the checkpoint into seg[0] (bucket layout), as asynchronous copies that
    // are all in flight together.
    {
      const float* in = ckpt + (inst * n_ckpt + kc) * (int64_t)N * N;
      for (int idx = lane; idx < C::MAT; idx += 32) seg[idx] = 0.f;
      __syncwarp();
      const int dq = 32 / N, dm = 32 % N;
      int r = lane / N, cc = lane % N;                 // (r, cc) of element e, advanced by 32
      for (int e = lane; e < N * N; e += 32) {
        const int br = r == N - 1 ? NB : r, bc = cc == N - 1 ? NB : cc;
        if (bc <= br && TASER_IN(tri_off(br) + bc, C::MAT) &&
            TASER_IN((inst * n_ckpt + kc) * N * N + e, batch * n_ckpt * N * N))
          uf_cp_async4(seg + tri_off(br) + bc, in + e);
        r += dq;
        cc += dm;
        if (cc >= N) { cc -= N; ++r; }
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncwarp();
    }
    // recompute L~(t0+1) .. L~(t1-1) into seg[1..]
    float l[NB + 1];
    for (int s = t0 + 1; s < t1; ++s) {
      float* Lin = seg + (s - 1 - t0) * C::MAT;
      float* Lout = seg + (TASER_IN(s - t0, c + 1) ? s - t0 : 0) * C::MAT;
      for (int idx = lane; idx < C::MAT; idx += 32) Lout[idx] = Lin[idx];  // zeros and L~_NN
      __syncwarp();
      if (j < NB) forward_step<NB>(Lin, Lout, l, tcol, alpha_t[s - 1] * inv, Dj, j);
      __syncwarp();
    }
    // reverse through steps t1 .. t0+1 (step s maps L~(s-1) -> L~(s), uses tau_{s})
    for (int s = t1; s > t0; --s) {
      const float* Lin = seg + (s - 1 - t0) * C::MAT;
      const float tau = alpha_t[s - 1] * inv;
      // G is not kept: taubar = <Vbar, G> = f (<G, Lbar> - rn proj <G, V>) (Lbar is zero
      // above the diagonal), so the two sums are taken while G is formed.
      float v[NB + 1];
      float gl = 0.f, gv = 0.f;
#pragma unroll
      for (int i = 0; i <= NB; ++i) {
        const float gi = (j < NB) ? 2.f * tri_row<NB>(Lin, i, tcol) : 0.f;
        v[i] = (i >= j && j < NB) ? fmaf(-tau, gi, Lin[tri_off(i) + (j < NB ? j : 0)]) : 0.f;
        gl = fmaf(gi, lbar[i], gl);
        gv = fmaf(gi, v[i], gv);
      }
      float n2 = 0.f;
#pragma unroll
      for (int i = 0; i <= NB; ++i) n2 = fmaf(v[i], v[i], n2);
      float proj = 0.f;
      const float rn = (n2 > 0.f && jr >= 0) ? rsqrtf(n2) : 0.f;
#pragma unroll
      for (int i = 0; i <= NB; ++i) proj = fmaf(v[i] * rn, lbar[i], proj);
      const float f = Dj * rn;
      // Vbar overwrites Lbar(s) in place.
#pragma unroll
      for (int i = 0; i <= NB; ++i) lbar[i] = (i >= j) ? f * fmaf(-v[i] * rn, proj, lbar[i]) : 0.f;
      const float tb = -warp_sum(f * fmaf(-rn * proj, gv, gl));
      if (lane == 0 && TASER_IN(inst * t_max + (s - 1), batch * t_max)) {
        grad_tau[inst * t_max + (s - 1)] = tb;
        TASER_FINITE(tb);
      }
      // Lbar(s-1) = tril(Vbar - tau Vbar (2 T~)): rows of Vbar through shared memory
#pragma unroll
      for (int i = 0; i <= NB; ++i)
        if (j < NB && i >= j) vb[tri_off(i) + j] = lbar[i];
      if (lane == 0) vb[tri_off(NB) + NB] = 0.f;   // column N of Vbar is zero
      __syncwarp();
#pragma unroll
      for (int i = 0; i <= NB; ++i) {
        const float p = 2.f * tri_row<NB>(vb, i, tcol);
        lbar[i] = (i >= j && j < NB) ? fmaf(-tau, p, lbar[i]) : 0.f;
      }
      __syncwarp();
    }
  }
}

// grad_alpha[t] = sum_n grad_tau[n][t] * inv_norm[n], one block per t, fixed-order tree.
__global__ void reduce_alpha_kernel(int64_t batch, int t_max, const float* __restrict__ grad_tau,
                                     const float* __restrict__ inv_norm, float* __restrict__ grad_alpha) {
  __shared__ float part[256];
  const int t = blockIdx.x;
  float acc = 0.f;
  for (int64_t n = threadIdx.x; n < batch; n += blockDim.x) acc = fmaf(grad_tau[n * t_max + t], inv_norm[n], acc);
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad_alpha[t] = part[0];
}

template <int NB>
static cudaError_t launch_unfolded(bool backward, int64_t batch, int N, const float* Tt, const float* D,
                                   const float* inv_norm, const float* alpha_t, int t_max, int c, float* ckpt,
                                   float* soft, int8_t* s_hat, const float* grad_soft, float* grad_tau,
                                   cudaStream_t st) {
  using C = UfCfg<NB>;
  const int64_t blocks = (batch + C::WARPS - 1) / C::WARPS;
  if (!backward) {
    const size_t smem = (size_t)C::WARPS * 2 * C::MAT * sizeof(float);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(unfolded_forward_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
    }
    unfolded_forward_kernel<NB><<<(unsigned)blocks, 128, smem, st>>>(batch, N, Tt, D, inv_norm, alpha_t, t_max, c,
                                                                     ckpt, soft, s_hat);
  } else {
    const size_t smem = (size_t)C::BWD_WARPS * (c + 2) * C::MAT * sizeof(float);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(unfolded_backward_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t bblocks = (batch + C::BWD_WARPS - 1) / C::BWD_WARPS;
    unfolded_backward_kernel<NB><<<(unsigned)bblocks, 32 * C::BWD_WARPS, smem, st>>>(
        batch, N, Tt, D, inv_norm, alpha_t, t_max, c, ckpt, grad_soft, grad_tau);
  }
  return cudaGetLastError();
}

// Shared memory the backward kernel needs for checkpoint spacing c at size N (bytes).
size_t unfolded_backward_smem(int N, int c) {
  const int NB = bucket_of(N);
  return (size_t)UfCfg<32>::BWD_WARPS * (c + 2) * tri_off(NB + 1) * sizeof(float);
}

cudaError_t unfolded_tc(bool backward, bool fp16, int64_t batch, int N, const float* Tt, const float* D,
                        const float* inv_norm, const float* alpha_t, int t_max, int c, float* ckpt, float* soft,
                        int8_t* s_hat, const float* grad_soft, float* grad_tau, cudaStream_t st);

// precision: TASER_FP32, or TASER_BF16_TC / TASER_FP16_TC (tensor-core kernels for bucket 32;
// smaller N runs the FP32 kernels).
cudaError_t unfolded(bool backward, int precision, int64_t batch, int N, const float* Tt, const float* D,
                     const float* inv_norm, const float* alpha_t, int t_max, int c, float* ckpt, float* soft,
                     int8_t* s_hat, const float* grad_soft, float* grad_tau, float* grad_alpha, cudaStream_t st) {
  cudaError_t e;
  const bool tc = precision != TASER_FP32 && bucket_of(N) == 32;
  switch (tc ? -1 : bucket_of(N)) {
    case -1:
      e = unfolded_tc(backward, precision == TASER_FP16_TC, batch, N, Tt, D, inv_norm, alpha_t, t_max, c, ckpt, soft,
                      s_hat, grad_soft, grad_tau, st);
      break;
    case 8:
      e = launch_unfolded<8>(backward, batch, N, Tt, D, inv_norm, alpha_t, t_max, c, ckpt, soft, s_hat, grad_soft,
                             grad_tau, st);
      break;
    case 16:
      e = launch_unfolded<16>(backward, batch, N, Tt, D, inv_norm, alpha_t, t_max, c, ckpt, soft, s_hat, grad_soft,
                              grad_tau, st);
      break;
    case 32:
      e = launch_unfolded<32>(backward, batch, N, Tt, D, inv_norm, alpha_t, t_max, c, ckpt, soft, s_hat, grad_soft,
                              grad_tau, st);
      break;
    default:
      return cudaErrorNotSupported;
  }
  if (e != cudaSuccess || !backward || grad_alpha == nullptr) return e;
  reduce_alpha_kernel<<<t_max, 256, 0, st>>>(batch, t_max, grad_tau, inv_norm, grad_alpha);
  return cudaGetLastError();
}

}  // namespace taser

TASER_DEBUG_COLLECTOR(unfolded)
