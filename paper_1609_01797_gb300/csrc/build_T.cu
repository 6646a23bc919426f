// Per-instance construction of T~ and D (Sec. II-A Eq. 2, Sec. II-B Eq. 5, Sec. III-C).
//
// T is never formed from the real-valued 2B x N matrices of the paper.  Both problem
// families only need the complex Gram matrix Gamma = X^H X of the B x M augmented matrix
// X = [H, y] (MIMO) or X = [Y_1 .. Y_{K-1}, Y_0] (JED, pilot moved last), because
//   Hbar^T Hbar = [[Re G, -Im G], [Im G, Re G]],  Hbar^T ybar = [Re z; Im z]   (QPSK)
//   Hunder^T Hunder = Re G,  Hunder^T ybar = Re z                               (BPSK, JED)
// with G = H^H H and z = H^H y.  Reading the complex input once, this halves the work
// of the real route and the B x M input is the only HBM traffic besides T~ and D.
//
// Mapping: one warp per instance.  X is staged in shared memory 128 (or 64) antennas at a
// time with cp.async; each lane takes whole antenna rows and accumulates a pass of 32 (or
// 16) Gram entries in registers (register-only FFMAs), then a 5-step transpose-reduce
// over the lanes leaves every lane with complete sums for one entry (or half of one).  Entries are
// enumerated cyclically (entry (a, d) is Gamma[a][(a + d) mod MP], d <= (MP-1)/2), which
// covers each unordered pair once.
#include "common.cuh"

namespace taser {

template <int MP>
struct BuildCfg {
  static constexpr int E = MP * (MP + 1) / 2;        // Gram entries
  static constexpr int DMAX = (MP - 1) / 2;
  static constexpr int SLOTS = MP <= 17 ? 32 : 16;   // entries per pass
  static constexpr int NVAL = 2 * SLOTS;             // floats reduced per pass
  static constexpr int PASSES = (E + SLOTS - 1) / SLOTS;
  static constexpr int CH = MP <= 17 ? 128 : 64;     // antennas per staged chunk
  static constexpr int RPL = CH / 32;                // antennas per lane per chunk
  static constexpr int WARPS = 4;
  static constexpr int X_FLOATS = CH * MP * 2;
  static constexpr int G_FLOATS = NVAL * PASSES;
  static constexpr int WARP_FLOATS = X_FLOATS + G_FLOATS;
  static constexpr int SMEM_BYTES = WARPS * WARP_FLOATS * 4;
};

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int MP>
__device__ __forceinline__ float2 gram_at(const float* Gs, int p, int q) {
  using C = BuildCfg<MP>;
  int d = q - p;
  if (d < 0) d += MP;
  if (d <= C::DMAX) {
    const int e = d * MP + p;
    return make_float2(Gs[2 * e], Gs[2 * e + 1]);
  }
  const int e = (MP - d) * MP + q;  // stored as Gamma[q][p] = conj(Gamma[p][q])
  return make_float2(Gs[2 * e], -Gs[2 * e + 1]);
}

// Real index a of T -> (complex column of X, part): part 0 = real, 1 = imaginary,
// 2 = the augmented column.
__device__ __forceinline__ void t_index(int kind, int a, int P, int MP, int& col, int& part) {
  if (kind == TASER_MIMO_QPSK) {
    if (a < P) { col = a; part = 0; }
    else if (a < 2 * P) { col = a - P; part = 1; }
    else { col = MP - 1; part = 2; }
  } else {
    if (a < P) { col = a; part = 0; }
    else { col = MP - 1; part = 2; }
  }
}

template <int MP>
__device__ __forceinline__ float t_entry(const float* Gs, int kind, int P, int a, int b) {
  int ca, pa, cb, pb;
  t_index(kind, a, P, MP, ca, pa);
  t_index(kind, b, P, MP, cb, pb);
  const float2 g = gram_at<MP>(Gs, ca, cb);
  if (kind == TASER_SIMO_JED_BPSK) return -g.x;
  if (kind == TASER_MIMO_BPSK) return (pa == 2) == (pb == 2) ? g.x : -g.x;
  // QPSK with the effective channel H / sqrt2.
  const float c = 0.70710678118654752f;
  if (pa == 2 && pb == 2) return g.x;
  if (pa == 2 || pb == 2) {
    // one augmented index: -c * (Re or Im) of Gamma[user][aug]
    const int pu = pa == 2 ? pb : pa;
    const float2 z = pa == 2 ? make_float2(g.x, -g.y) : g;  // Gamma[user][aug]
    return -c * (pu == 0 ? z.x : z.y);
  }
  if (pa == pb) return 0.5f * g.x;
  return pa == 0 ? -0.5f * g.y : 0.5f * g.y;
}

template <int MP>
__global__ void __launch_bounds__(128)
build_T_kernel(int kind, int64_t batch, int B, int P, int N, const float2* __restrict__ X,
               const float2* __restrict__ yv, float* __restrict__ Tt, float* __restrict__ Dout,
               uint32_t* __restrict__ flags) {
  using C = BuildCfg<MP>;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t inst = (int64_t)blockIdx.x * C::WARPS + warp;
  if (inst >= batch) return;
  float* Xs = smem + warp * C::WARP_FLOATS;
  float* Gs = Xs + C::X_FLOATS;
  float2* Xc = reinterpret_cast<float2*>(Xs);

  for (int i = lane; i < C::G_FLOATS; i += 32) Gs[i] = 0.f;
  // Padding columns P..MP-2 stay zero for the whole kernel.
  if (P < MP - 1) {
    for (int i = lane; i < C::CH * MP; i += 32) Xc[i] = make_float2(0.f, 0.f);
  }
  const bool jed = kind == TASER_SIMO_JED_BPSK;
  const int src_cols = jed ? P + 1 : P;                 // columns per antenna row in X
  const float2* Xi = X + inst * (int64_t)B * src_cols;
  const float2* yi = jed ? nullptr : yv + inst * (int64_t)B;
  // lane -> (row offset, column) for the staging copy
  const int rows_per_iter = P <= 32 ? 32 / P : 1;
  const int cr = lane / P, cc = lane % P;

  for (int r0 = 0; r0 < B; r0 += C::CH) {
    const int rows = min(C::CH, B - r0);
    __syncwarp();
    if (rows < C::CH) {
      for (int i = rows * MP + lane; i < C::CH * MP; i += 32) Xc[i] = make_float2(0.f, 0.f);
    }
    // Stage X[r0 .. r0+rows) into padded rows of MP complex values.
    if (P <= 32) {
      if (cr < rows_per_iter) {
        for (int r = cr; r < rows; r += rows_per_iter) {
          const float2* src = Xi + (int64_t)(r0 + r) * src_cols + (jed ? cc + 1 : cc);
          cp_async8(&Xc[r * MP + cc], src);
        }
      }
    }
    for (int r = lane; r < rows; r += 32) {
      const float2* src = jed ? Xi + (int64_t)(r0 + r) * src_cols : yi + (r0 + r);
      cp_async8(&Xc[r * MP + MP - 1], src);
    }
    cp_async_wait_all();
    __syncwarp();

    const int nrr = (rows + 31) >> 5;  // antenna rows per lane in this chunk
#pragma unroll
    for (int pass = 0; pass < C::PASSES; ++pass) {
      float acc[C::NVAL];
#pragma unroll
      for (int i = 0; i < C::NVAL; ++i) acc[i] = 0.f;
#pragma unroll 1
      for (int rr = 0; rr < nrr; ++rr) {
        const float2* xr = Xc + (lane + 32 * rr) * MP;
        float2 x[MP];
#pragma unroll
        for (int c = 0; c < MP; ++c) x[c] = xr[c];  // unused columns are dead loads
#pragma unroll
        for (int s = 0; s < C::SLOTS; ++s) {
          const int e = pass * C::SLOTS + s;  // compile-time after unrolling
          if (e < C::E) {
            const int a = e % MP, d = e / MP;
            const int b = (a + d) % MP;
            // conj(x_a) x_b
            acc[2 * s] = fmaf(x[a].x, x[b].x, fmaf(x[a].y, x[b].y, acc[2 * s]));
            if (d != 0) acc[2 * s + 1] = fmaf(x[a].x, x[b].y, fmaf(-x[a].y, x[b].x, acc[2 * s + 1]));
          }
        }
      }
      // Transpose-reduce over lane bits 4..0 (bit 4 first, keeping the upper half when
      // the bit is set): the lane ends with values [off, off + NVAL/32), off = (NVAL/32) * lane.
#pragma unroll
      for (int step = 0; step < 5; ++step) {
        const int m = 16 >> step;
        const int h = C::NVAL >> (step + 1);
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
          const float send = up ? acc[i] : acc[i + h];
          const float keep = up ? acc[i + h] : acc[i];
          acc[i] = keep + __shfl_xor_sync(TASER_FULL_MASK, send, m);
        }
      }
      constexpr int PER = C::NVAL / 32;
#pragma unroll
      for (int q = 0; q < PER; ++q) Gs[pass * C::NVAL + PER * lane + q] += acc[q];
    }
  }
  __syncwarp();

  // D_a = sqrt|T_aa| (1 where T_aa == 0) and the flags.
  uint32_t fl = 0;
  float* Dsm = Xs;  // reuse the staging buffer: D then 1/D
  float* rDsm = Xs + 128;
  for (int a = lane; a < N; a += 32) {
    const float taa = t_entry<MP>(Gs, kind, P, a, a);
    if (!isfinite(taa)) fl |= TASER_FLAG_NONFINITE;
    float da = sqrtf(fabsf(taa));
    if (taa == 0.f) {
      da = 1.f;
      fl |= TASER_FLAG_ZERO_DIAG;
    }
    Dsm[a] = da;
    rDsm[a] = 1.f / da;
    Dout[inst * N + a] = da;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fl |= __shfl_xor_sync(TASER_FULL_MASK, fl, o);
  if (lane == 0 && flags != nullptr) flags[inst] = fl;
  __syncwarp();
  float* To = Tt + inst * (int64_t)N * N;
  for (int a = 0; a < N; ++a) {
    const float ra = rDsm[a];
    for (int b = lane; b < N; b += 32) {
      const float tab = t_entry<MP>(Gs, kind, P, a, b);
      float v;
      if (a == b) {
        v = tab > 0.f ? 1.f : (tab < 0.f ? -1.f : 0.f);
      } else {
        v = tab * ra * rDsm[b];
      }
      To[(int64_t)a * N + b] = v;
    }
  }
}

template <int MP>
static cudaError_t launch_build(int kind, int64_t batch, int B, int P, int N, const float2* X, const float2* y,
                                float* Tt, float* D, uint32_t* flags, cudaStream_t st) {
  using C = BuildCfg<MP>;
  cudaError_t e = cudaFuncSetAttribute(build_T_kernel<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       C::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (batch + C::WARPS - 1) / C::WARPS;
  build_T_kernel<MP><<<(unsigned)blocks, 32 * C::WARPS, C::SMEM_BYTES, st>>>(kind, batch, B, P, N, X, y, Tt, D,
                                                                           flags);
  return cudaGetLastError();
}

// P = data columns (U for MIMO, K-1 for JED); the augmented column sits at MP-1.
cudaError_t build_T(int kind, int64_t batch, int B, int P, int N, const void* X, const void* y, float* Tt,
                    float* D, uint32_t* flags, cudaStream_t st) {
  const float2* Xc = static_cast<const float2*>(X);
  const float2* yc = static_cast<const float2*>(y);
  if (P + 1 <= 9) return launch_build<9>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
  if (P + 1 <= 17) return launch_build<17>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
  if (P + 1 <= 33) return launch_build<33>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
  return cudaErrorNotSupported;
}

}  // namespace taser
