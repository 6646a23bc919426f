// Per-instance construction of T~ and D (Sec. II-A Eq. 2, Sec. II-B Eq. 5, Sec. III-C).
//
// T is never formed from the real-valued 2B x N matrices of the paper.  Both problem
// families only need the complex Gram matrix Gamma = X^H X of the B x M augmented matrix
// X = [H, y] (MIMO) or X = [Y_1 .. Y_{K-1}, Y_0] (JED, pilot moved last), because
//   Hbar^T Hbar = [[Re G, -Im G], [Im G, Re G]],  Hbar^T ybar = [Re z; Im z]   (QPSK)
//   Hunder^T Hunder = Re G,  Hunder^T ybar = Re z                               (BPSK, JED)
// with G = H^H H and z = H^H y.  The complex input is read once; it is the only HBM
// traffic besides the T~ and D outputs.
//
// Gamma comes from the real Gram G' = W^T W of W = X viewed as B x 2M floats (real and
// imaginary parts interleaved, exactly the complex64 memory layout):
//   Re Gamma_pq = G'[2p][2q] + G'[2p+1][2q+1],   Im Gamma_pq = G'[2p][2q+1] - G'[2p+1][2q].
// G' is a dense contraction over the B antennas, so it runs on the tensor cores with
// mma.sync m16n8k16 FP16 (FP32 accumulation) in the split form x = hi + lo (hi = fp16(x),
// lo = fp16(x - hi)), G' = hi^T hi + hi^T lo + lo^T hi, which keeps FP32-level accuracy
// (relative error about 2^-22 per product) while the reduction over B happens inside the
// tensor core.  FP16's range is met by a power-of-two scale per column of W (exact, undone
// on G'), taken from the first 32 antenna rows with 2^8 of headroom; an overflow restarts
// the instance at a smaller scale.
//
// Mapping: one warp per instance.  X is staged into shared memory in chunks of antenna rows,
// by the tensor memory accelerator (cp.async.bulk.tensor into an mbarrier ring) for QPSK with
// 16 users and an even B, by a per-lane cp.async ring otherwise; only the upper-triangular
// 16 x 8 tiles of G' are computed.
#include <cuda.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"

namespace taser {

template <int MP>
struct BuildCfg {
  static constexpr int NCR = 2 * MP;                  // real columns of W
  static constexpr int NT = (NCR + 7) / 8;            // n-tiles of 8 columns
  static constexpr int MT = (NCR + 15) / 16;          // m-tiles of 16 columns
  // Row stride (floats) of a staged antenna row: >= 8 NT and = 8 or 24 mod 32, so the
  // fragment loads (rows t and t + 4, columns 8j + g) hit 32 distinct banks.
  static constexpr int WS = (8 * NT) % 32 == 8 || (8 * NT) % 32 == 24 ? 8 * NT : 8 * NT + 8;
  // Staging: a ring of NS chunks of CH antenna rows.  17 complex columns (the QPSK 128x16
  // case) use 16-row chunks with three in flight; the others a double buffer of 32 rows
  // (measured: the deeper ring was slower for 33 columns).
  static constexpr int CH = MP == 17 ? 16 : 32;       // antennas per staged chunk
  static constexpr int NS = MP == 17 ? 4 : 2;         // chunks in the cp.async ring
  static constexpr int BUF_FLOATS = CH * WS;
  static constexpr int WARPS = 4;
  static constexpr int WARP_FLOATS = NS * BUF_FLOATS; // ring; reused by the epilogue
  static constexpr int SMEM_BYTES = WARPS * WARP_FLOATS * 4;
  // FP16 split Gram (m16n8k16) from 17 complex columns on; 3xTF32 (m16n8k8) below, where
  // the scale search costs more than the faster tensor rate saves (measured).
  static constexpr bool F16 = MP >= 17;
  __host__ __device__ static constexpr bool tile(int i, int j) { return j >= 2 * i && j < NT; }
};
// The Gram loop's shared-memory reads use compile-time offsets: rows below CH of a chunk,
// columns below 8 NT, and (scale search) rows below 32 of the first two chunks.
static_assert((BuildCfg<9>::CH - 1) * BuildCfg<9>::WS + 8 * BuildCfg<9>::NT <= BuildCfg<9>::BUF_FLOATS, "");
static_assert((BuildCfg<17>::CH - 1) * BuildCfg<17>::WS + 8 * BuildCfg<17>::NT <= BuildCfg<17>::BUF_FLOATS, "");
static_assert((BuildCfg<33>::CH - 1) * BuildCfg<33>::WS + 8 * BuildCfg<33>::NT <= BuildCfg<33>::BUF_FLOATS, "");
static_assert(31 * BuildCfg<17>::WS + 8 * BuildCfg<17>::NT <= 2 * BuildCfg<17>::BUF_FLOATS, "");

// The BPSK kinds need only Re Gamma' (T = +-A^T A with A = [Re; Im] stacked), which is the
// Gram of the real rows: each antenna row contributes its real and its imaginary part as two
// k-rows, and the columns are the complex columns themselves.  Against the interleaved
// complex Gram that is half the columns, a quarter of the tiles and half the MMAs, and a
// k-row pair (Re, Im) is one 8-byte shared-memory read.  Used with the FP16 split (MP >= 17).
template <int MP>
struct RealGramCfg {
  static constexpr int NT = (MP + 7) / 8;             // n-tiles of 8 columns
  static constexpr int MT = (MP + 15) / 16;           // m-tiles of 16 columns
  __host__ __device__ static constexpr bool tile(int i, int j) { return j >= 2 * i && j < NT; }
};
// The real-row reads stay inside a staged row: column c < MP is floats 2c, 2c + 1.
static_assert(2 * 17 <= BuildCfg<17>::WS && 2 * 33 <= BuildCfg<33>::WS, "");
template <int MP, int KIND>
__host__ __device__ constexpr bool real_gram() {
  return MP >= 17 && (KIND == TASER_MIMO_BPSK || KIND == TASER_SIMO_JED_BPSK);
}
static_assert(31 * BuildCfg<33>::WS + 8 * BuildCfg<33>::NT <= BuildCfg<33>::BUF_FLOATS, "");

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NLEFT>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NLEFT) : "memory"); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Scales a pair of floats of one column by sc2 = {2^e, 2^e} (exact) and splits it into FP16
// high and low parts: x = hi + lo + O(2^-22 x).  The scaling and the residual x - hi run as
// packed f32x2 operations.
__device__ __forceinline__ void split_f16(float x0, float x1, uint64_t sc2, uint32_t& hi, uint32_t& lo) {
  const uint64_t xs = f2mul(f2pack(x0, x1), sc2);
  float a, b;
  f2unpack(xs, a, b);
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  float r0, r1;
  f2unpack(f2fma(f2pack(hf.x, hf.y), f2pack(-1.f, -1.f), xs), r0, r1);
  const __half2 l = __floats2half2_rn(r0, r1);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// An int known at compile time, usable where a runtime int is expected.
template <int V>
struct CInt {
  __host__ __device__ constexpr operator int() const { return V; }
};

// 2^e as a float for -126 <= e <= 127.
__device__ __forceinline__ float pow2i(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Staging by the tensor memory accelerator (TMA).  QPSK problems that fill the column
// bucket (16 users: 17 complex columns with y) stage their antenna rows with
// cp.async.bulk.tensor instead of per-lane cp.async.  H is a 3-D tensor (32 floats per
// antenna row, B rows, batch instances) read in boxes of 16 rows with the 128-byte swizzle;
// rows past B read as zero.  y is a 2-D tensor (2B floats per instance) read in boxes of 32
// floats.  One lane per warp arms a stage's mbarrier with the expected bytes and issues both
// copies; every lane waits on the barrier's phase.  Each wait is bounded by a clock64
// budget.  An expired wait marks the instance TASER_FLAG_TIMEOUT, waits (bounded again) for
// the warp's other copies in flight and leaves that instance's T~ and D unwritten.
struct TmaCfg {
  static constexpr int NS = 4;                        // stages in the ring
  static constexpr int H_FLOATS = 16 * 32;            // one H box: 16 rows of 128 bytes
  static constexpr int Y_FLOATS = 32;                 // one y box: 16 complex values
  static constexpr unsigned TX_BYTES = (H_FLOATS + Y_FLOATS) * 4;
  static constexpr int WARP_FLOATS = 2304;            // NS (H + y) = 2,176 floats, in 1 KB units
  static constexpr int WARPS = 4;
  // Per block: the warps' rings, their mbarriers and 1 KB of slack to align the rings.
  static constexpr int SMEM_BYTES = WARPS * WARP_FLOATS * 4 + WARPS * NS * 8 + 1024;
};
static_assert(TmaCfg::NS * (TmaCfg::H_FLOATS + TmaCfg::Y_FLOATS) <= TmaCfg::WARP_FLOATS, "ring must fit");
static_assert((TmaCfg::WARP_FLOATS * 4) % 1024 == 0, "swizzled boxes need 1 KB alignment");
static_assert(33 * 33 + 3 + 144 <= TmaCfg::WARP_FLOATS, "epilogue scratch (tile, its offset, D) must fit the ring");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// Arrives once and adds `tx` bytes to the phase's expected transaction count.
__device__ __forceinline__ void mbar_arm(uint32_t bar, unsigned tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for the completion of the phase with the given parity; false once `budget` clock
// cycles have passed without it.  A phase that has already completed costs one test and
// no clock read.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

#ifdef TASER_DEBUG
// Debug build only: the staging copy of chunk g_drop_chunk of instance g_drop_inst is
// withheld, so that its bounded wait expires (the timeout path under test).
static __device__ long long g_drop_inst = -1;
static __device__ int g_drop_chunk = -1;
#endif

// KIND >= 0 compiles the epilogue for that problem kind; -1 takes it from kind_rt.
// TMA: staging by the tensor memory accelerator (MP = 17, QPSK only; see TmaCfg).
template <int MP, int KIND, bool TMA = false>
__global__ void __launch_bounds__(128, MP == 17 ? 5 : (real_gram<MP, KIND>() ? 3 : 1))
build_T_kernel(int kind_rt, int64_t batch, int B, int P, int N, const float2* __restrict__ X,
               const float2* __restrict__ yv, float* __restrict__ Tt, float* __restrict__ Dout,
               uint32_t* __restrict__ flags, const __grid_constant__ CUtensorMap tmH,
               const __grid_constant__ CUtensorMap tmY, long long wait_budget) {
  using C = BuildCfg<MP>;                      // staging (and the interleaved complex Gram)
  constexpr bool REAL = real_gram<MP, KIND>();
  using GT = std::conditional_t<REAL, RealGramCfg<MP>, BuildCfg<MP>>;   // Gram tiles
  constexpr int NT = GT::NT, MT = GT::MT, WS = C::WS, CH = C::CH;
  constexpr int WFL = TMA ? TmaCfg::WARP_FLOATS : C::WARP_FLOATS;   // floats per warp
  static_assert(!TMA || (MP == 17 && KIND == TASER_MIMO_QPSK), "TMA staging serves the 17-column QPSK Gram");
  const int kind = KIND >= 0 ? KIND : kind_rt;
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int64_t inst = (int64_t)blockIdx.x * C::WARPS + warp;
  if (inst >= batch) return;
  float* sbase = smem;
  if constexpr (TMA) {   // swizzled boxes start on 1 KB boundaries
    const uint32_t a = smem_u32(smem);
    sbase = smem + ((((a + 1023u) & ~1023u) - a) >> 2);
  }
  float* Ws = sbase + warp * WFL;

  if constexpr (!TMA) {
    // Padding columns (2P .. 2MP-3 and >= 2MP) stay zero for the whole Gram phase.
    for (int i = lane; i < C::WARP_FLOATS / 4; i += 32)
      reinterpret_cast<float4*>(Ws)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
  }
  const bool jed = kind == TASER_SIMO_JED_BPSK || kind == TASER_SIMO_JED_QPSK;
  const int src_cols = jed ? P + 1 : P;                 // complex columns per antenna row
  const float2* Xi = X + inst * (int64_t)B * src_cols;
  const float2* yi = jed ? nullptr : yv + inst * (int64_t)B;
  const bool pairs = !jed && (P % 2 == 0) && ((reinterpret_cast<uintptr_t>(Xi) & 15) == 0);
  const int units = pairs ? P / 2 : P;                  // copy units per antenna row
  const int rows_per_iter = units <= 32 ? 32 / units : 1;
  const int crow = lane / units, cu = lane % units;
  const int nchunks = (B + CH - 1) / CH;

  auto stage = [&](int chunk) {
    float* buf = Ws + (chunk % C::NS) * C::BUF_FLOATS;
    const int r0 = chunk * CH;
    const int rows = min(CH, B - r0);
    if (crow < rows_per_iter) {
      for (int r = crow; r < rows; r += rows_per_iter) {
        [[maybe_unused]] const int64_t xe = (inst * B + r0 + r) * src_cols;   // element of the row in X
        const float2* src = Xi + (int64_t)(r0 + r) * src_cols;
        if (pairs) {
          if (TASER_IN(r * WS + 4 * cu + 3, C::BUF_FLOATS) && TASER_IN(xe + 2 * cu + 1, batch * B * src_cols))
            cp_async16(buf + r * WS + 4 * cu, src + 2 * cu);
        } else {
          const int sc = jed ? cu + 1 : cu;
          if (TASER_IN(r * WS + 2 * cu + 1, C::BUF_FLOATS) && TASER_IN(xe + sc, batch * B * src_cols))
            cp_async8(buf + r * WS + 2 * cu, src + sc);
        }
      }
    }
    for (int r = lane; r < rows; r += 32) {
      const float2* src = jed ? Xi + (int64_t)(r0 + r) * src_cols : yi + (r0 + r);
      [[maybe_unused]] const int64_t se = jed ? (inst * B + r0 + r) * src_cols : inst * B + r0 + r;
      if (TASER_IN(r * WS + 2 * (MP - 1) + 1, C::BUF_FLOATS) && TASER_IN(se, batch * B * (jed ? src_cols : 1)))
        cp_async8(buf + r * WS + 2 * (MP - 1), src);
    }
    cp_async_commit();
  };

  float acc[MT][NT][4];
  // Exponent e_q of the power-of-two scale of complex column q = 4j + tq (FP16 Gram only):
  // the accumulators hold Gamma'_pq = 2^(e_p + e_q) Gamma_pq.
  int exq[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) exq[j] = 0;
  // Real-row Gram: exponent of column q = 8j + 2tq + e of this lane's accumulators.
  [[maybe_unused]] int exr[NT][2];
  if constexpr (TMA) {
    // The FP16-split Gram of the branch below (same scales, restart and tiles), staged by
    // TMA.  A 16-row step pairs rows (2tq, 2tq + 1) and (2tq + 8, 2tq + 9) as its k-indices;
    // under the 128-byte swizzle, row r's float c lives at r 32 + ((c / 4) ^ (r mod 8)) 4 +
    // c mod 4, and these rows put the 32 lanes of every fragment load in 32 banks.
    using TC = TmaCfg;
    float* const Hs = Ws;                          // NS boxes of 16 x 32 floats (swizzled)
    float* const Ys = Ws + TC::NS * TC::H_FLOATS;  // NS boxes of 32 floats
    uint64_t* const bars = reinterpret_cast<uint64_t*>(sbase + TC::WARPS * TC::WARP_FLOATS) + warp * TC::NS;
    if (lane == 0) {
      for (int st = 0; st < TC::NS; ++st) mbar_init(smem_u32(bars + st), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // Chunks are numbered across restarts: chunk sequence q sits in stage q mod NS, and its
    // barrier phase has parity (q / NS) mod 2.
    unsigned q_issued = 0;
    auto issue = [&](int chunk) {   // called by every lane; lane 0 arms and copies
      const unsigned q = q_issued++;
      if (lane != 0) return;
#ifdef TASER_DEBUG
      if (inst == g_drop_inst && chunk == g_drop_chunk) return;   // withheld (timeout test)
#endif
      const int st = (int)(q % TC::NS);
      const uint32_t bar = smem_u32(bars + st);
      mbar_arm(bar, TC::TX_BYTES);
      tma_load_3d(smem_u32(Hs + st * TC::H_FLOATS), &tmH, 0, chunk * 16, (int)inst, bar);
      tma_load_2d(smem_u32(Ys + st * TC::Y_FLOATS), &tmY, chunk * 32, (int)inst, bar);
    };
    auto arrived = [&](unsigned q) -> bool {
      const bool ok = mbar_wait(smem_u32(bars + q % TC::NS), (q / TC::NS) & 1u, wait_budget);
      return __all_sync(TASER_FULL_MASK, ok);
    };
    // Per-lane parts of the swizzled addresses: row 2tq (+8) and row 2tq + 1 (+9) of column
    // 8j + g are at base0 / base1 + 8 (j ^ tq) (+ 256).
    const int gb = g >> 2, gi = g & 3;
    const int base0 = 64 * tq + 4 * gb + gi, base1 = 64 * tq + 32 + 4 * (gb ^ 1) + gi, t8 = 8 * tq;
    const bool ylane = g < 2;                      // n-tile 4: column 32 + g is y (re, im) for g < 2
    int ex[NT];
    float sc[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) ex[j] = 0;
    bool timed_out = false;
    unsigned q_fail = 0;
    for (int attempt = 0; attempt < 16 && !timed_out; ++attempt) {
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
      const unsigned q0 = q_issued;
#pragma unroll
      for (int st = 0; st < TC::NS - 1; ++st)
        if (st < nchunks) issue(st);
      for (int chunk = 0; chunk < nchunks; ++chunk) {
        const unsigned q = q0 + chunk;
        if (!arrived(q)) {
          timed_out = true;
          q_fail = q;
          break;
        }
        if (attempt == 0 && chunk == 0) {
          // Column maxima over the first 32 antenna rows (chunks 0 and 1; rows past B read
          // as zero), then over tq and over the re / im pair of a complex column.
          if (nchunks > 1 && !arrived(q + 1)) {
            timed_out = true;
            q_fail = q + 1;
            break;
          }
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            float m = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              if (h == 1 && nchunks < 2) continue;
              const float* hb = Hs + ((q + h) % TC::NS) * TC::H_FLOATS;
              const float* yb = Ys + ((q + h) % TC::NS) * TC::Y_FLOATS;
              if (j < 4) {
                const int x = (8 * j) ^ t8;
                m = fmaxf(m, fmaxf(fmaxf(fabsf(hb[base0 + x]), fabsf(hb[base1 + x])),
                                   fmaxf(fabsf(hb[base0 + x + 256]), fabsf(hb[base1 + x + 256]))));
              } else if (ylane) {
                m = fmaxf(m, fmaxf(fmaxf(fabsf(yb[4 * tq + g]), fabsf(yb[4 * tq + 2 + g])),
                                   fmaxf(fabsf(yb[4 * tq + 16 + g]), fabsf(yb[4 * tq + 18 + g]))));
              }
            }
            m = fmaxf(m, __shfl_xor_sync(TASER_FULL_MASK, m, 1));
            m = fmaxf(m, __shfl_xor_sync(TASER_FULL_MASK, m, 2));
            m = fmaxf(m, __shfl_xor_sync(TASER_FULL_MASK, m, 4));   // re and im of one column
            const int e2 = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;
            ex[j] = (m > 0.f && e2 > -127) ? min(max(6 - e2, -100), 100) : 0;
          }
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) sc[j] = pow2i(ex[j]);
        // Chunk c + NS - 1 goes into the stage of chunk c - 1, which every lane has read.
        if (chunk + TC::NS - 1 < nchunks) issue(chunk + TC::NS - 1);
        const float* hb = Hs + (q % TC::NS) * TC::H_FLOATS;
        const float* yb = Ys + (q % TC::NS) * TC::Y_FLOATS;
        uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          const uint64_t sc2 = f2pack(sc[j], sc[j]);
          float x0, x1, x2, x3;
          if (j < 4) {
            const int x = (8 * j) ^ t8;
            x0 = hb[base0 + x];
            x1 = hb[base1 + x];
            x2 = hb[base0 + x + 256];
            x3 = hb[base1 + x + 256];
          } else {
            x0 = ylane ? yb[4 * tq + g] : 0.f;
            x1 = ylane ? yb[4 * tq + 2 + g] : 0.f;
            x2 = ylane ? yb[4 * tq + 16 + g] : 0.f;
            x3 = ylane ? yb[4 * tq + 18 + g] : 0.f;
          }
          split_f16(x0, x1, sc2, bh[j][0], bl[j][0]);
          split_f16(x2, x3, sc2, bh[j][1], bl[j][1]);
        }
#pragma unroll
        for (int i = 0; i < MT; ++i) {
          // A = W^T: rows 16i + g (+8) are n-tiles 2i and 2i+1 of the same loads.
          const int j0 = 2 * i, j1 = 2 * i + 1;
          uint32_t ah[4], al[4];
          ah[0] = bh[j0][0];
          ah[2] = bh[j0][1];
          al[0] = bl[j0][0];
          al[2] = bl[j0][1];
          if (j1 < NT) {
            ah[1] = bh[j1][0];
            ah[3] = bh[j1][1];
            al[1] = bl[j1][0];
            al[3] = bl[j1][1];
          } else {
            ah[1] = ah[3] = al[1] = al[3] = 0u;
          }
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            if (!GT::tile(i, j)) continue;
            mma_f16(acc[i][j], ah, bh[j][0], bh[j][1]);
            mma_f16(acc[i][j], ah, bl[j][0], bl[j][1]);
            mma_f16(acc[i][j], al, bh[j][0], bh[j][1]);
          }
        }
        __syncwarp();  // every lane has read this stage before it is refilled
      }
      if (timed_out) break;
      bool finite = true;
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) finite = finite && isfinite(acc[i][j][e]);
      if (__all_sync(TASER_FULL_MASK, finite)) break;   // no FP16 overflow (non-finite input retries)
#pragma unroll
      for (int j = 0; j < NT; ++j) ex[j] -= 9;
    }
    if (timed_out) {
      // Wait (bounded) for every copy of this warp that may still be in flight, so that
      // none lands in shared memory after the warp has left; then flag the instance.
      for (unsigned q = q_fail; q < q_issued; ++q) (void)arrived(q);
      if (lane == 0 && flags != nullptr && TASER_IN(inst, batch)) flags[inst] = TASER_FLAG_TIMEOUT;
      return;
    }
#pragma unroll
    for (int j = 0; j < NT; ++j) exq[j] = __shfl_sync(TASER_FULL_MASK, ex[j], 4 * (2 * tq));
  } else if constexpr (REAL) {
    // The FP16-split Gram of the real rows (BPSK kinds): same per-column power-of-two scales,
    // restart and tiles as the complex branch below.  A 16-row k-step takes 8 antenna rows:
    // k-rows 2tq and 2tq + 1 are the real and imaginary parts of staged row tq, k-rows
    // 2tq + 8 and 2tq + 9 those of row tq + 4, so each B register is one (Re, Im) pair of
    // column 8j + g.  Columns >= MP read as zero.
    int ex[NT];
    float sc[NT];
  #pragma unroll
    for (int j = 0; j < NT; ++j) ex[j] = 0;
    for (int attempt = 0; attempt < 16; ++attempt) {
  #pragma unroll
      for (int i = 0; i < MT; ++i)
  #pragma unroll
        for (int j = 0; j < NT; ++j)
  #pragma unroll
          for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  #pragma unroll
      for (int s = 0; s < C::NS - 1; ++s) {
        if (s < nchunks) stage(s); else cp_async_commit();
      }
      for (int chunk = 0; chunk < nchunks; ++chunk) {
        cp_async_wait<C::NS - 2>();
        __syncwarp();
        float* buf = Ws + (chunk % C::NS) * C::BUF_FLOATS;
        const int rows = min(CH, B - chunk * CH);
        if (rows < CH) {  // zero the unused tail rows of the last chunk
          for (int i = rows * WS + lane; i < CH * WS; i += 32) buf[i] = 0.f;
          __syncwarp();
        }
        if (attempt == 0 && chunk == 0) {
          // Column maxima over the first 32 antenna rows (rows past B read as zero): the real
          // and imaginary parts of rows tq + 4r of column 8j + g, then over tq.
          if constexpr (CH < 32) {
            static_assert(CH == 16 && C::NS >= 3, "the first 32 rows must be chunks 0 and 1");
            cp_async_wait<C::NS - 3>();
            __syncwarp();
            if (nchunks > 1 && B - CH < CH) {
              float* b1 = Ws + C::BUF_FLOATS;
              for (int i = (B - CH) * WS + lane; i < CH * WS; i += 32) b1[i] = 0.f;
              __syncwarp();
            }
          }
  #pragma unroll
          for (int j = 0; j < NT; ++j) {
            float m = 0.f;
            if (8 * j + g < MP) {
  #pragma unroll
              for (int r = 0; r < 32 / 4; ++r) {
                const float2 v = *reinterpret_cast<const float2*>(Ws + (tq + 4 * r) * WS + 2 * (8 * j + g));
                m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
              }
            }
            m = fmaxf(m, __shfl_xor_sync(TASER_FULL_MASK, m, 1));
            m = fmaxf(m, __shfl_xor_sync(TASER_FULL_MASK, m, 2));
            const int e2 = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;   // floor(log2 m), m normal
            ex[j] = (m > 0.f && e2 > -127) ? min(max(6 - e2, -100), 100) : 0;
          }
        }
  #pragma unroll
        for (int j = 0; j < NT; ++j) sc[j] = pow2i(ex[j]);
        if (chunk + C::NS - 1 < nchunks) stage(chunk + C::NS - 1); else cp_async_commit();
  #pragma unroll
        for (int ks = 0; ks < CH / 8; ++ks) {
          uint32_t bh[NT][2], bl[NT][2];
          const float* rp = buf + (8 * ks + tq) * WS + 2 * g;
  #pragma unroll
          for (int j = 0; j < NT; ++j) {
            const uint64_t sc2 = f2pack(sc[j], sc[j]);
            float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
            if (8 * j + g < MP) {
              v0 = *reinterpret_cast<const float2*>(rp + 16 * j);
              v1 = *reinterpret_cast<const float2*>(rp + 4 * WS + 16 * j);
            }
            split_f16(v0.x, v0.y, sc2, bh[j][0], bl[j][0]);
            split_f16(v1.x, v1.y, sc2, bh[j][1], bl[j][1]);
          }
  #pragma unroll
          for (int i = 0; i < MT; ++i) {
            // A = W^T: rows 16i + g (+8) are n-tiles 2i and 2i+1 of the same loads.
            const int j0 = 2 * i, j1 = 2 * i + 1;
            uint32_t ah[4], al[4];
            ah[0] = bh[j0][0];
            ah[2] = bh[j0][1];
            al[0] = bl[j0][0];
            al[2] = bl[j0][1];
            if (j1 < NT) {
              ah[1] = bh[j1][0];
              ah[3] = bh[j1][1];
              al[1] = bl[j1][0];
              al[3] = bl[j1][1];
            } else {
              ah[1] = ah[3] = al[1] = al[3] = 0u;
            }
  #pragma unroll
            for (int j = 0; j < NT; ++j) {
              if (!GT::tile(i, j)) continue;
              mma_f16(acc[i][j], ah, bh[j][0], bh[j][1]);
              mma_f16(acc[i][j], ah, bl[j][0], bl[j][1]);
              mma_f16(acc[i][j], al, bh[j][0], bh[j][1]);
            }
          }
        }
        __syncwarp();  // every lane has read this buffer before it is refilled
      }
      bool finite = true;
  #pragma unroll
      for (int i = 0; i < MT; ++i)
  #pragma unroll
        for (int j = 0; j < NT; ++j)
  #pragma unroll
          for (int e = 0; e < 4; ++e) finite = finite && isfinite(acc[i][j][e]);
      if (__all_sync(TASER_FULL_MASK, finite)) break;   // no FP16 overflow (non-finite input retries)
  #pragma unroll
      for (int j = 0; j < NT; ++j) ex[j] -= 9;
    }
    // Column q = 8j + 2tq + e of the accumulators is column 8j + g of lane g = 2tq + e.
  #pragma unroll
    for (int j = 0; j < NT; ++j) {
      exr[j][0] = __shfl_sync(TASER_FULL_MASK, ex[j], 4 * (2 * tq));
      exr[j][1] = __shfl_sync(TASER_FULL_MASK, ex[j], 4 * (2 * tq + 1));
    }
  } else if constexpr (C::F16) {
    // Per-column power-of-two scales: this lane's columns 8j + g are multiplied by 2^ex[j]
    // before the FP16 split, chosen from the first 32 antenna rows so that the largest
    // magnitude of the complex column (its real and imaginary parts share one scale) lands in
    // [2^6, 2^7).  A later value beyond FP16's range (65504) becomes an infinite high part and
    // a non-finite accumulator; the whole Gram then restarts with every scale 2^-9 smaller.
    // Sharing the scale within a complex column makes Gamma'_pq = 2^(e_p + e_q) Gamma_pq, so
    // the normalised T~_pq = Gamma'_pq / (D'_p D'_q) needs no unscaling (the powers of two
    // cancel exactly) and only D_p = D'_p 2^-e_p does.
    int ex[NT];
    float sc[NT];
  #pragma unroll
    for (int j = 0; j < NT; ++j) ex[j] = 0;
    for (int attempt = 0; attempt < 16; ++attempt) {
  #pragma unroll
      for (int i = 0; i < MT; ++i)
  #pragma unroll
        for (int j = 0; j < NT; ++j)
  #pragma unroll
          for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
      // One cp.async group per chunk (empty past the end), so the wait for chunk c always
      // leaves the NS - 2 younger groups in flight; chunk c + NS - 1 is issued before chunk
      // c is consumed (into the buffer of chunk c - 1), so NS - 1 chunks load during the MMAs.
  #pragma unroll
      for (int s = 0; s < C::NS - 1; ++s) {
        if (s < nchunks) stage(s); else cp_async_commit();
      }
      for (int chunk = 0; chunk < nchunks; ++chunk) {
        cp_async_wait<C::NS - 2>();
        __syncwarp();
        float* buf = Ws + (chunk % C::NS) * C::BUF_FLOATS;
        const int rows = min(CH, B - chunk * CH);
        if (rows < CH) {  // zero the unused tail rows of the last chunk
          for (int i = rows * WS + lane; i < CH * WS; i += 32) buf[i] = 0.f;
          __syncwarp();
        }
        if (attempt == 0 && chunk == 0) {
          // Column maxima over the first 32 antenna rows (rows past B read as zero): rows
          // tq + 4r of column 8j + g, then over tq.  With 16-row chunks these are chunks 0
          // and 1, which sit next to each other at the start of the ring.
          if constexpr (CH < 32) {
            static_assert(CH == 16 && C::NS >= 3, "the first 32 rows must be chunks 0 and 1");
            cp_async_wait<C::NS - 3>();
            __syncwarp();
            if (nchunks > 1 && B - CH < CH) {
              float* b1 = Ws + C::BUF_FLOATS;
              for (int i = (B - CH) * WS + lane; i < CH * WS; i += 32) b1[i] = 0.f;
              __syncwarp();
            }
          }
  #pragma unroll
          for (int j = 0; j < NT; ++j) {
            float m = 0.f;
  #pragma unroll
            for (int r = 0; r < 32 / 4; ++r) m = fmaxf(m, fabsf(Ws[(tq + 4 * r) * WS + 8 * j + g]));
            m = fmaxf(m, __shfl_xor_sync(TASER_FULL_MASK, m, 1));
            m = fmaxf(m, __shfl_xor_sync(TASER_FULL_MASK, m, 2));
            m = fmaxf(m, __shfl_xor_sync(TASER_FULL_MASK, m, 4));   // re and im of one column
            const int e2 = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;   // floor(log2 m), m normal
            ex[j] = (m > 0.f && e2 > -127) ? min(max(6 - e2, -100), 100) : 0;
          }
        }
  #pragma unroll
        for (int j = 0; j < NT; ++j) sc[j] = pow2i(ex[j]);
        if (chunk + C::NS - 1 < nchunks) stage(chunk + C::NS - 1); else cp_async_commit();
  #pragma unroll
        for (int ks = 0; ks < CH / 16; ++ks) {
          // B fragments of n-tile j: k = 2tq, 2tq+1, 2tq+8, 2tq+9 are staged rows tq, tq+4,
          // tq+8, tq+12 of this 16-row step (any fixed row order gives the same Gram), column
          // 8j + g; each value is scaled and split into FP16 high and low parts.
          uint32_t bh[NT][2], bl[NT][2];
          const float* rp = buf + (16 * ks + tq) * WS + g;
  #pragma unroll
          for (int j = 0; j < NT; ++j) {
            const uint64_t sc2 = f2pack(sc[j], sc[j]);
            split_f16(rp[8 * j], rp[4 * WS + 8 * j], sc2, bh[j][0], bl[j][0]);
            split_f16(rp[8 * WS + 8 * j], rp[12 * WS + 8 * j], sc2, bh[j][1], bl[j][1]);
          }
  #pragma unroll
          for (int i = 0; i < MT; ++i) {
            // A = W^T: rows 16i + g (+8) are n-tiles 2i and 2i+1 of the same loads.
            const int j0 = 2 * i, j1 = 2 * i + 1;
            uint32_t ah[4], al[4];
            ah[0] = bh[j0][0];
            ah[2] = bh[j0][1];
            al[0] = bl[j0][0];
            al[2] = bl[j0][1];
            if (j1 < NT) {
              ah[1] = bh[j1][0];
              ah[3] = bh[j1][1];
              al[1] = bl[j1][0];
              al[3] = bl[j1][1];
            } else {
              ah[1] = ah[3] = al[1] = al[3] = 0u;
            }
  #pragma unroll
            for (int j = 0; j < NT; ++j) {
              if (!GT::tile(i, j)) continue;
              mma_f16(acc[i][j], ah, bh[j][0], bh[j][1]);
              mma_f16(acc[i][j], ah, bl[j][0], bl[j][1]);
              mma_f16(acc[i][j], al, bh[j][0], bh[j][1]);
            }
          }
        }
        __syncwarp();  // every lane has read this buffer before it is refilled
      }
      bool finite = true;
  #pragma unroll
      for (int i = 0; i < MT; ++i)
  #pragma unroll
        for (int j = 0; j < NT; ++j)
  #pragma unroll
          for (int e = 0; e < 4; ++e) finite = finite && isfinite(acc[i][j][e]);
      if (__all_sync(TASER_FULL_MASK, finite)) break;   // no FP16 overflow (non-finite input retries)
  #pragma unroll
      for (int j = 0; j < NT; ++j) ex[j] -= 9;
    }
    // The exponent of complex column q = 4j + tq is that of its real column 2q = 8j + 2tq.
#pragma unroll
    for (int j = 0; j < NT; ++j) exq[j] = __shfl_sync(TASER_FULL_MASK, ex[j], 4 * (2 * tq));
  } else {   // 3xTF32 on m16n8k8: no range handling needed, cheaper for few columns
  #pragma unroll
    for (int i = 0; i < MT; ++i)
  #pragma unroll
      for (int j = 0; j < NT; ++j)
  #pragma unroll
        for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    stage(0);
    if (nchunks > 1) stage(1);
    for (int chunk = 0; chunk < nchunks; ++chunk) {
      if (chunk + 1 < nchunks) cp_async_wait<1>(); else cp_async_wait<0>();
      __syncwarp();
      float* buf = Ws + (chunk & 1) * C::BUF_FLOATS;
      const int rows = min(CH, B - chunk * CH);
      if (rows < CH) {  // zero the unused tail rows of the last chunk
        for (int i = rows * WS + lane; i < CH * WS; i += 32) buf[i] = 0.f;
        __syncwarp();
      }
  #pragma unroll
      for (int ks = 0; ks < CH / 8; ++ks) {
        // B fragments of every n-tile (k = 8 ks + tq, 8 ks + tq + 4; column 8j + g), split.
        uint32_t bh[NT][2], bl[NT][2];
        const float* r0p = buf + (8 * ks + tq) * WS + g;
        const float* r1p = r0p + 4 * WS;
  #pragma unroll
        for (int j = 0; j < NT; ++j) {
          const float x0 = r0p[8 * j], x1 = r1p[8 * j];
          bh[j][0] = to_tf32(x0);
          bh[j][1] = to_tf32(x1);
          bl[j][0] = to_tf32(x0 - __uint_as_float(bh[j][0]));
          bl[j][1] = to_tf32(x1 - __uint_as_float(bh[j][1]));
        }
  #pragma unroll
        for (int i = 0; i < MT; ++i) {
          // A = W^T: rows 16i + g (+8) are n-tiles 2i and 2i+1 of the same loads.
          const int j0 = 2 * i, j1 = 2 * i + 1;
          uint32_t ah[4], al[4];
          ah[0] = bh[j0][0];
          ah[2] = bh[j0][1];
          al[0] = bl[j0][0];
          al[2] = bl[j0][1];
          if (j1 < NT) {
            ah[1] = bh[j1][0];
            ah[3] = bh[j1][1];
            al[1] = bl[j1][0];
            al[3] = bl[j1][1];
          } else {
            ah[1] = ah[3] = al[1] = al[3] = 0u;
          }
  #pragma unroll
          for (int j = 0; j < NT; ++j) {
            if (!GT::tile(i, j)) continue;
            mma_tf32(acc[i][j], ah, bh[j][0], bh[j][1]);
            mma_tf32(acc[i][j], ah, bl[j][0], bl[j][1]);
            mma_tf32(acc[i][j], al, bh[j][0], bh[j][1]);
          }
        }
      }
      __syncwarp();  // every lane has read this buffer
      if (chunk + 2 < nchunks) stage(chunk + 2);
    }
  }

  // Gamma_pq (p <= q) from the accumulators: lane (g, tq) holds rows 16i + g (+8) and
  // columns 8j + 2tq, +1 of G', i.e. complex column q = 4j + tq; rows 2p and 2p+1 of
  // complex row p sit in lanes g and g + 1 (even g combines).  Each (p, q) with p <= q
  // lies in exactly one computed tile.
  // (The real-row Gram holds Re Gamma'_pq directly: row p = 16i + g (+8), column
  // q = 8j + 2tq (+1) of each tile.)
  [[maybe_unused]] float gre[MT][NT][2], gim[MT][NT][2];
  if constexpr (!REAL) {
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        if (!GT::tile(i, j)) continue;
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = __shfl_xor_sync(TASER_FULL_MASK, acc[i][j][e], 4);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          gre[i][j][h] = acc[i][j][2 * h] + o[2 * h + 1];
          gim[i][j][h] = acc[i][j][2 * h + 1] - o[2 * h];
        }
      }
  }
  const bool holder = (g & 1) == 0;
  // Complex column p -> real indices of T: (ire, iim, kind of column) with the augmented
  // column last.  QPSK user p: real p and U + p; BPSK / JED data column p: real p.
  const bool qpsk = kind == TASER_MIMO_QPSK || kind == TASER_SIMO_JED_QPSK;
  const bool jq = kind == TASER_SIMO_JED_QPSK;
  float* Dc = Ws + WFL - 2 * 72;              // D per complex column
  float* rDc = Dc + 72;                       // 1 / D per complex column
  float* Ts = Ws;                             // N x N staging of T~ (reuses the buffers)
  __syncwarp();
  // Diagonal: D and the flags.
  uint32_t fl = 0;
  if constexpr (REAL) {
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        if (!GT::tile(i, j)) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int p = 16 * i + g + 8 * h, q = 8 * j + 2 * tq + e;
            if (p == q && (p < P || p == MP - 1)) {
              const float v = acc[i][j][2 * h + e];
              const float taa = fabsf(v);                 // 2^(2 e_p) |T_pp|
              if (!isfinite(v)) fl |= TASER_FLAG_NONFINITE;
              float da = sqrtf(taa);                      // D'_p = 2^e_p D_p
              float dtrue = ldexpf(da, -exr[j][e]);
              if (taa == 0.f) {
                da = 1.f;
                dtrue = 1.f;
                fl |= TASER_FLAG_ZERO_DIAG;
              }
              if (TASER_IN(p, 72)) {
                Dc[p] = dtrue;
                rDc[p] = 1.f / da;
              }
            }
          }
      }
  }
#pragma unroll
  for (int i = 0; i < MT && !REAL; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      if (!GT::tile(i, j)) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = 8 * i + 4 * h + (g >> 1), q = 4 * j + tq;
        if (holder && p == q && (p < P || p == MP - 1)) {
          const bool aug = p == MP - 1;
          const float taa = fabsf(gre[i][j][h]) * (qpsk && !aug ? 0.5f : 1.f);   // 2^(2 e_p) |T_pp|
          if (!isfinite(gre[i][j][h])) fl |= TASER_FLAG_NONFINITE;
          float da = sqrtf(taa);                                                  // D'_p = 2^e_p D_p
          float dtrue = ldexpf(da, -exq[j]);
          if (taa == 0.f) {
            da = 1.f;
            dtrue = 1.f;
            fl |= TASER_FLAG_ZERO_DIAG;
          }
          if (TASER_IN(p, 72)) {
            Dc[p] = dtrue;
            rDc[p] = 1.f / da;
          }
        }
      }
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fl |= __shfl_xor_sync(TASER_FULL_MASK, fl, o);
  if (lane == 0 && flags != nullptr && TASER_IN(inst, batch)) flags[inst] = fl;
  __syncwarp();
  // Off-diagonal and diagonal entries of T~ into the staging tile, then a coalesced copy of
  // T~ and D to global memory.  NU = users / data columns, Nr = N.  A QPSK problem that
  // fills the column bucket (U = MP - 1, e.g. 128x16) runs this with both as compile-time
  // constants, so every address of the scatter is a lane base plus an immediate offset.
  const float dsg = jed ? -1.f : 1.f;   // sign of T_aa
  auto scatter_and_store = [&](auto nu_c, auto nr_c) {
    const int NU = nu_c, Nr = nr_c;
    // The tile starts `mis` floats into the staging area, mis = (address of the instance's
    // T~ / 4) mod 4, so that its 16-byte groups coincide in shared and global memory and
    // the copy-out runs as 16-byte loads and stores between a scalar head and tail.
    float* To = Tt + inst * (int64_t)Nr * Nr;
    const int mis = (int)((reinterpret_cast<uintptr_t>(To) >> 2) & 3u);
    float* Tsm = Ts + mis;
    // Tsm[a] = v (a debug build checks a against the N x N tile).
    auto put = [&](int a, float v) {
      if (TASER_IN(a, Nr * Nr)) Tsm[a] = v;
    };
    if constexpr (REAL) {
      // BPSK kinds: T~_pq = T~_qp = +-Re Gamma'_pq / (D'_p D'_q), the augmented column last.
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          if (!GT::tile(i, j)) continue;
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int p = 16 * i + g + 8 * h, q = 8 * j + 2 * tq + e;
              const bool pv = p < NU, qv = q < NU, qa = q == MP - 1, pa = p == MP - 1;
              if (p > q || !(pv || pa) || !(qv || qa)) continue;
              const float re = acc[i][j][2 * h + e];
              const float sc = (TASER_IN(p, 72) && TASER_IN(q, 72)) ? rDc[p] * rDc[q] : 0.f;
              const int ap = pa ? Nr - 1 : p, aq = qa ? Nr - 1 : q;
              if (p == q) {
                put(ap * Nr + ap, re == 0.f ? 0.f : dsg);
                continue;
              }
              // MIMO BPSK: A = [H, -y] flips the sign of the augmented column's entries;
              // JED BPSK: T = -A^T A.
              const float v = (kind == TASER_SIMO_JED_BPSK ? -re : (qa ? -re : re)) * sc;
              put(ap * Nr + aq, v);
              put(aq * Nr + ap, v);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < MT && !REAL; ++i)
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        if (!GT::tile(i, j)) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int p = 8 * i + 4 * h + (g >> 1), q = 4 * j + tq;
          const bool pv = p < NU, qv = q < NU, qa = q == MP - 1, pa = p == MP - 1;
          if (!holder || p > q || !(pv || pa) || !(qv || qa)) continue;
          const float re = gre[i][j][h], im = gim[i][j][h];
          const float sc = (TASER_IN(p, 72) && TASER_IN(q, 72)) ? rDc[p] * rDc[q] : 0.f;
          const int ap = pa ? Nr - 1 : p, aq = qa ? Nr - 1 : q;     // real index of the Re part
          if (p == q) {
            const float dv = re == 0.f ? 0.f : dsg;
            put(ap * Nr + ap, dv);
            if (qpsk && !pa) {
              put((NU + p) * Nr + (NU + p), dv);
              put(p * Nr + (NU + p), 0.f);
              put((NU + p) * Nr + p, 0.f);
            }
            continue;
          }
          if (kind == TASER_SIMO_JED_BPSK) {
            const float v = -re * sc;
            put(ap * Nr + aq, v);
            put(aq * Nr + ap, v);
          } else if (kind == TASER_MIMO_BPSK) {
            const float v = (qa ? -re : re) * sc;
            put(ap * Nr + aq, v);
            put(aq * Nr + ap, v);
          } else if (qa) {
            // user p with the augmented column: -c [Re z; Im z].  JED QPSK: the pilot column
            // is y_0 s_0 with s_0 = (1 + j)/sqrt2, so z = s_0 (Y_r^H y_0) (and A = [Hbar, +ybar]
            // with T = -A^T A gives the same sign as MIMO's A = [Hbar, -ybar], T = A^T A).
            const float c = 0.70710678118654752f;
            const float zr = jq ? c * (re - im) : re, zi = jq ? c * (re + im) : im;
            const float vr = -c * zr * sc, vi = -c * zi * sc;
            put(p * Nr + aq, vr);
            put(aq * Nr + p, vr);
            put((NU + p) * Nr + aq, vi);
            put(aq * Nr + (NU + p), vi);
          } else {
            // users p < q: [[Re G, -Im G], [Im G, Re G]] / 2 (negated for JED: T = -A^T A)
            const float hh = jq ? -0.5f : 0.5f;
            const float vr = hh * re * sc, vi = hh * im * sc;
            put(p * Nr + q, vr);
            put(q * Nr + p, vr);
            put((NU + p) * Nr + (NU + q), vr);
            put((NU + q) * Nr + (NU + p), vr);
            put(p * Nr + (NU + q), -vi);
            put((NU + q) * Nr + p, -vi);
            put((NU + p) * Nr + q, vi);
            put(q * Nr + (NU + p), vi);
          }
        }
      }
    __syncwarp();
    const int e0 = (4 - mis) & 3;                 // first entry on a 16-byte boundary
    const int nvec = (Nr * Nr - e0) >> 2;
    const int e1 = e0 + 4 * nvec;                 // first entry of the scalar tail
    if (lane < e0 || (lane >= 4 && lane - 4 < Nr * Nr - e1)) {
      const int e = lane < e0 ? lane : e1 + lane - 4;
      if (TASER_IN(inst * Nr * Nr + e, batch * Nr * Nr)) To[e] = Tsm[e];
      TASER_FINITE(Tsm[e]);
    }
    const float4* src4 = reinterpret_cast<const float4*>(Tsm + e0);
    float4* dst4 = reinterpret_cast<float4*>(To + e0);
    for (int v = lane; v < nvec; v += 32) {
      const float4 x = src4[v];
      if (TASER_IN(inst * Nr * Nr + e0 + 4 * v + 3, batch * Nr * Nr)) dst4[v] = x;
      TASER_FINITE(x.x);
      TASER_FINITE(x.y);
      TASER_FINITE(x.z);
      TASER_FINITE(x.w);
    }
    for (int a = lane; a < Nr; a += 32) {
      const int p = a == Nr - 1 ? MP - 1 : (qpsk && a >= NU ? a - NU : a);
      if (TASER_IN(inst * Nr + a, batch * Nr) && TASER_IN(p, 72)) {
        Dout[inst * Nr + a] = Dc[p];
        TASER_FINITE(Dc[p]);
      }
    }
  };
  if (qpsk && P == MP - 1 && N == 2 * MP - 1) {
    scatter_and_store(CInt<MP - 1>{}, CInt<2 * MP - 1>{});
  } else {
    scatter_and_store(P, N);
  }
}

template <int MP, int KIND>
static cudaError_t launch_build(int kind, int64_t batch, int B, int P, int N, const float2* X, const float2* y,
                                float* Tt, float* D, uint32_t* flags, cudaStream_t st) {
  using C = BuildCfg<MP>;
  static_assert((2 * MP - 1) * (2 * MP - 1) + 3 + 144 <= C::WARP_FLOATS,
                "epilogue scratch (tile, its offset, D) must fit the staging buffers");
  if (C::SMEM_BYTES > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(build_T_kernel<MP, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (batch + C::WARPS - 1) / C::WARPS;
  const CUtensorMap unused{};
  build_T_kernel<MP, KIND><<<(unsigned)blocks, 32 * C::WARPS, C::SMEM_BYTES, st>>>(kind, batch, B, P, N, X, y, Tt,
                                                                                 D, flags, unused, unused, 0);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link-time dependency on
// the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// Bound on one staging wait of the TMA kernel, in SM clock cycles (about a second).
constexpr long long kTmaWaitCycles = 1ll << 31;

// QPSK with 16 users through the TMA kernel.  The tensor maps need 16-byte aligned bases
// (the ABI requires them), byte strides that are multiples of 16 (B even) and 32-bit
// coordinates.  Returns cudaErrorNotSupported when the problem does not qualify.
static cudaError_t launch_build_tma(int64_t batch, int B, const float2* X, const float2* y, float* Tt, float* D,
                                    uint32_t* flags, cudaStream_t st) {
  const EncodeTiledFn encode = encode_tiled();
  if (encode == nullptr || B % 2 != 0 || batch > (int64_t)INT32_MAX || (int64_t)B * 16 > (int64_t)INT32_MAX ||
      (reinterpret_cast<uintptr_t>(X) & 15u) != 0 || (reinterpret_cast<uintptr_t>(y) & 15u) != 0)
    return cudaErrorNotSupported;
  CUtensorMap mh, my;
  const cuuint64_t hdim[3] = {32, (cuuint64_t)B, (cuuint64_t)batch};
  const cuuint64_t hstride[2] = {128, (cuuint64_t)B * 128};
  const cuuint32_t hbox[3] = {32, 16, 1}, one[3] = {1, 1, 1};
  CUresult r = encode(&mh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(X), hdim, hstride, hbox, one,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const cuuint64_t ydim[2] = {(cuuint64_t)B * 2, (cuuint64_t)batch};
  const cuuint64_t ystride[1] = {(cuuint64_t)B * 8};
  const cuuint32_t ybox[2] = {32, 1};
  r = encode(&my, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(y), ydim, ystride, ybox, one,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int64_t blocks = (batch + TmaCfg::WARPS - 1) / TmaCfg::WARPS;
  build_T_kernel<17, TASER_MIMO_QPSK, true><<<(unsigned)blocks, 32 * TmaCfg::WARPS, TmaCfg::SMEM_BYTES, st>>>(
      TASER_MIMO_QPSK, batch, B, 16, 33, X, y, Tt, D, flags, mh, my, kTmaWaitCycles);
  return cudaGetLastError();
}

#ifdef TASER_DEBUG
// Debug build: withhold the staging copy of `chunk` of instance `inst` in later TMA launches
// (inst < 0: none).
cudaError_t debug_drop_copy(int64_t inst, int chunk) {
  const long long i = inst;
  cudaError_t e = cudaMemcpyToSymbol(g_drop_inst, &i, sizeof(i));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_drop_chunk, &chunk, sizeof(chunk));
  return e;
}
#endif

// P = data columns (U for MIMO, K-1 for JED); the augmented column sits at MP-1.
cudaError_t build_T(int kind, int64_t batch, int B, int P, int N, const void* X, const void* y, float* Tt,
                    float* D, uint32_t* flags, cudaStream_t st) {
  const float2* Xc = static_cast<const float2*>(X);
  const float2* yc = static_cast<const float2*>(y);
  if (P + 1 <= 9) return launch_build<9, -1>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
  if (P + 1 <= 17) {
    if (kind == TASER_MIMO_QPSK && P == 16) {
      const cudaError_t e = launch_build_tma(batch, B, Xc, yc, Tt, D, flags, st);
      if (e != cudaErrorNotSupported) return e;
    }
    if (kind == TASER_MIMO_QPSK)
      return launch_build<17, TASER_MIMO_QPSK>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
    if (kind == TASER_MIMO_BPSK)   // the BPSK kinds: Gram of the real rows
      return launch_build<17, TASER_MIMO_BPSK>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
    if (kind == TASER_SIMO_JED_BPSK)
      return launch_build<17, TASER_SIMO_JED_BPSK>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
    return launch_build<17, -1>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
  }
  if (P + 1 <= 33) {
    if (kind == TASER_MIMO_BPSK)
      return launch_build<33, TASER_MIMO_BPSK>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
    if (kind == TASER_SIMO_JED_BPSK)
      return launch_build<33, TASER_SIMO_JED_BPSK>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
    return launch_build<33, -1>(kind, batch, B, P, N, Xc, yc, Tt, D, flags, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace taser

TASER_DEBUG_COLLECTOR(build_T)
