// Gradient pass of the envelope formula on tcgen05 tensor cores (squared-Euclidean cost,
// bf16-rounded points, the problem LAMP_PREC_BF16_TC solves):
//
//   dL/dx_i = 2 s (r_i x_i - q_i sum_j P_ij y_j),     P_ij  = 2^{v_ij} w_j
//   dL/dy_j = 2 s (A_j y_j - w_j sum_i P'_ji x_i),    P'_ji = 2^{v_ij} q_i
//
// with X_ij = q_i 2^{v_ij} w_j the coupling of the state's X^t (v the compensated exponent
// of stream A that the sweeps evaluate, q_i = r_i / S_i, w_j the column factor, A = col(X^t)).
// One pass per side recomputes X on the fly and never stores it: a CTA keeps 128 points of
// one side fixed and streams 64-point tiles of the other; per streamed tile
//   MMA 1:  S = x_fixed . y_tile^T            (M = 128, N = 64, K = 64 coordinates) -> TMEM
//   epilogue: P = 2^{v} w from S (one ex2 per entry), split into bf16 P_hi + P_lo (the pair
//             carries 16 significant bits) and stored to TMEM as the A operand of
//   MMA 2:  O += P_hi . yT_tile^T + P_lo . yT_tile^T   (M = 128, N = 64 coordinates,
//             K = 64 streamed points) into an FP32 accumulator that stays in TMEM over the
//             CTA's whole range of streamed tiles.
// yT is a transposed bf16 copy of the streamed points (64 coordinates x points), so both
// MMAs read K-major 128-byte-swizzled tiles written by TMA.  The CTA writes its O rows as
// float32 partials per inner split; k_tc_grad_fin adds the splits as a float-float pair and
// forms the gradient in float-float arithmetic (one float64 conversion per point: this
// part's FP64 rate is a small fraction of its FP32 rate).
//
// CTA = 10 warps: warps 0-7 epilogue (warp w: TMEM lanes 32 (w % 4) .. + 31, i.e. one fixed
// point per thread, and streamed columns [32 (w / 4), + 32)), warp 8 TMA producer, warp 9
// MMA issuer.  TMEM: three 64-column buffers, each holding S of a tile and then, written by
// the epilogue over the S it has read, P_hi and P_lo of that tile (MMA 2's A operand), and
// O (64 columns): 256.  The epilogue thus never waits for MMA 2: MMA 1 of tile i + 3 waits
// until MMA 2 of tile i has read its buffer, and the issuer runs MMA 1 two tiles ahead of
// MMA 2 (S of tile i + 2 is issued before P of tile i is awaited).
// Every mbarrier wait is bounded; on timeout the kernel records LAMP_E_TIMEOUT, stops
// issuing, waits (bounded) for its own copies and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "lamp_async.cuh"
#include "lamp_common.cuh"
#include "lamp_tc.cuh"

namespace lamp {
namespace tcg {

using namespace tc;
using async::bulk_load;
using async::fence_proxy_async_smem;
using async::mbar_arrive;
using async::mbar_drain;
using async::mbar_expect_tx;
using async::mbar_init;
using async::tma_load_2d;

constexpr int kTile = 128;                      // fixed points per CTA = M of both MMAs
constexpr int kStream = 64;                     // streamed points per tile = N of MMA 1 = K of MMA 2
constexpr int kK = 64;                          // padded coordinates = K of MMA 1 = N of MMA 2
constexpr int kStages = 4;                      // streamed-tile ring (points + transposed points)
constexpr int kTileBytes = kTile * kK * 2;      // 16 KiB
constexpr int kStreamBytes = kStream * kK * 2;  // 8 KiB per streamed tile, same for its transpose
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kSliceCols = 32;  // streamed columns of one epilogue warp
constexpr int kProducerWarp = kEpiWarps;
constexpr int kMmaWarp = kEpiWarps + 1;
constexpr int kThreads = (kEpiWarps + 2) * 32;
constexpr uint32_t kTmemCols = 256;
constexpr int kBufs = 3;          // S / P buffers of 64 columns each
constexpr uint32_t kColO = kBufs * kStream;  // O accumulator: 64 FP32 columns
static_assert(kEpiWarps == 8 && kStream == 2 * kSliceCols, "epilogue layout: 4 lane quadrants x 2 slices");

struct __align__(8) Bars {
  uint64_t fixed_full;
  uint64_t full[kStages];   // points tile and transposed tile of a ring slot landed
  uint64_t empty[kStages];  // both MMAs of the slot's tile done
  uint64_t s_full[kBufs];   // MMA 1 wrote S into a buffer
  uint64_t p_full[kBufs];   // the epilogue replaced it by P_hi, P_lo
  uint64_t buf_free[kBufs]; // MMA 2 read P: the buffer takes the next S
  uint64_t o_full;          // the last MMA 2 completed: O is final
  uint64_t drain;           // error path: every MMA issued so far completed
  uint64_t pair_full[2];    // packed offsets / weights of a streamed tile landed (bulk copy)
  uint64_t pair_empty[2];
  uint32_t tmem_base;
  int err;
};
constexpr int kBarBytes = 256;
static_assert(sizeof(Bars) <= kBarBytes, "barrier block");

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, Bars* B, DevState* dev) {
  return async::mbar_wait(bar, parity, &B->err, dev, async::kWaitLimit);
}

// D[tmem] (+)= A[tmem] * B[smem]^T, kind::f16: the A operand (M x K bf16) is read from TMEM,
// lane = row, two bf16 per 32-bit column (the lower k in the low half)
__device__ __forceinline__ void umma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 8 FP32 columns of this warp's 32 lanes (no wait)
__device__ __forceinline__ void tmem_ld8(uint32_t ta, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(ta)
               : "memory");
}

__device__ __forceinline__ void tmem_wait_ld8(uint32_t (&v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
               :
               : "memory");
}

// 16 consecutive 32-bit columns of this warp's 32 lanes from registers
__device__ __forceinline__ void tmem_st16(uint32_t ta, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(ta),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// 8 consecutive 32-bit columns of this warp's 32 lanes from registers
__device__ __forceinline__ void tmem_st8(uint32_t ta, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(ta), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 32 FP32 columns of this warp's 32 lanes, waited for
__device__ __forceinline__ void tmem_ld32_wait(uint32_t ta, float (&out)[32]) {
  uint32_t v[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(ta)
      : "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) out[q] = __uint_as_float(v[q]);
}

// two floats -> bf16x2 with round-to-nearest-even: lo in bits 0-15, hi in bits 16-31
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// ROWS = true: dx side (fixed x points, streamed y tiles; weights w_j inside P, q_i after)
// ROWS = false: dy side (fixed y points, streamed x tiles; weights q_i inside P, w_j after)
// map_fixed: 128-row boxes of the fixed points; map_stream: 64-row boxes of the streamed
// points; map_streamT: 64 x 64 boxes of the transposed streamed points (64 x n_pad)
template <bool ROWS>
__global__ void __launch_bounds__(kThreads, 2)
k_tc_grad(const __grid_constant__ CUtensorMap map_fixed, const __grid_constant__ CUtensorMap map_stream,
          const __grid_constant__ CUtensorMap map_streamT, const Work w, int64_t n, int64_t m, int tiles_per_split,
          float* __restrict__ part, const Consts k) {
  DevState* __restrict__ dev = w.dev;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sFixed = smem;                               // 16 KiB
  unsigned char* sStream = smem + kTileBytes;                 // kStages x 8 KiB (points)
  unsigned char* sStreamT = sStream + kStages * kStreamBytes;  // kStages x 8 KiB (transposed)
  Bars* B = reinterpret_cast<Bars*>(sStreamT + kStages * kStreamBytes);
  float4* sPair = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(B) + kBarBytes);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int cur = dev->cur;
  const int64_t nfixed = ROWS ? n : m;
  const int64_t nstream = ROWS ? m : n;
  const int64_t fixed0 = (int64_t)blockIdx.x * kTile;
  const int64_t ntiles_all = (nstream + kStream - 1) / kStream;
  const int64_t it0 = (int64_t)blockIdx.y * tiles_per_split;
  int64_t it1 = it0 + tiles_per_split;
  if (it1 > ntiles_all) it1 = ntiles_all;
  const int ntiles = it1 > it0 ? (int)(it1 - it0) : 0;

  if (threadIdx.x == 0) {
    mbar_init(&B->fixed_full, 1);
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&B->full[s], 1);
      mbar_init(&B->empty[s], 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(&B->s_full[b], 1);
      mbar_init(&B->p_full[b], kEpiThreads);
      mbar_init(&B->buf_free[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&B->pair_full[b], 1);
      mbar_init(&B->pair_empty[b], kEpiThreads);
    }
    mbar_init(&B->o_full, 1);
    mbar_init(&B->drain, 1);
    B->err = 0;
    async::mbar_init_fence();
  }
  if (warp == 0) {
    tmem_alloc(&B->tmem_base, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = B->tmem_base;

  if (warp == kProducerWarp) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && ntiles > 0) {
      const float4* __restrict__ pair_src = ROWS ? w.colq2[cur] : w.g2row2;
      int issued = 0, pissued = 0;
      mbar_expect_tx(&B->fixed_full, kTileBytes);
      tma_load_2d(sFixed, &map_fixed, &B->fixed_full, 0, (int)fixed0);
      for (int i = 0; i < ntiles; ++i) {
        const int s = i % kStages;
        const int b = i & 1;
        const int row0 = (int)((it0 + i) * kStream);
        if (i >= kStages && !mbar_wait(&B->empty[s], ((i / kStages) & 1) ^ 1, B, dev)) break;
        mbar_expect_tx(&B->full[s], 2 * kStreamBytes);
        tma_load_2d(sStream + s * kStreamBytes, &map_stream, &B->full[s], 0, row0);
        tma_load_2d(sStreamT + s * kStreamBytes, &map_streamT, &B->full[s], row0, 0);
        issued = i + 1;
        if (i >= 2 && !mbar_wait(&B->pair_empty[b], ((i >> 1) - 1) & 1, B, dev)) break;
        mbar_expect_tx(&B->pair_full[b], kStream * sizeof(float4));
        bulk_load(sPair + (size_t)b * kStream, pair_src + (it0 + i) * kStream, kStream * sizeof(float4),
                  &B->pair_full[b]);
        pissued = i + 1;
      }
      if (*(volatile int*)&B->err) {
        mbar_drain(&B->fixed_full, 0);
        for (int i = issued - kStages < 0 ? 0 : issued - kStages; i < issued; ++i)
          mbar_drain(&B->full[i % kStages], (i / kStages) & 1);
        for (int i = pissued - 2 < 0 ? 0 : pissued - 2; i < pissued; ++i) mbar_drain(&B->pair_full[i & 1], (i >> 1) & 1);
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && ntiles > 0) {
      const uint32_t idesc = idesc_bf16(kTile, kStream);  // M = 128, N = 64 for both MMAs
      const uint32_t sF = smem_u32(sFixed);
      bool any = false;
      if (mbar_wait(&B->fixed_full, 0, B, dev)) {
        // MMA 1 of tile i into buffer i % kBufs: S = x_fixed . stream_i^T; it runs two tiles
        // ahead of MMA 2, so S of the tile after next is ready while the epilogue works
        auto mma1 = [&](int i) -> bool {
          const int s = i % kStages;
          const int b = i % kBufs;
          if (!mbar_wait(&B->full[s], (i / kStages) & 1, B, dev)) return false;
          if (i >= kBufs && !mbar_wait(&B->buf_free[b], ((i / kBufs) - 1) & 1, B, dev)) return false;
          tc_fence_after();
          const uint32_t sS = smem_u32(sStream + s * kStreamBytes);
#pragma unroll
          for (int kk = 0; kk < kK / 16; ++kk)
            umma_bf16(tmem + b * kStream, sdesc_sw128(sF + kk * 32), sdesc_sw128(sS + kk * 32), idesc, kk > 0);
          umma_commit(&B->s_full[b]);
          any = true;
          return true;
        };
        bool go = mma1(0) && (ntiles < 2 || mma1(1));
        for (int j = 0; go && j < ntiles; ++j) {
          if (j + 2 < ntiles && !mma1(j + 2)) break;
          // MMA 2 of tile j: O += P_hi . streamT_j^T + P_lo . streamT_j^T
          const int sj = j % kStages;
          const int bj = j % kBufs;
          if (!mbar_wait(&B->p_full[bj], (j / kBufs) & 1, B, dev)) break;
          tc_fence_after();
          const uint32_t sT = smem_u32(sStreamT + sj * kStreamBytes);
          // P of streamed points [16 kk, 16 kk + 16): slice kk / 2, half kk % 2 of the buffer
          // (8 columns of P_hi, then 8 of P_lo)
          const uint32_t pb = tmem + bj * kStream;
#pragma unroll
          for (int kk = 0; kk < kStream / 16; ++kk)
            umma_bf16_ts(tmem + kColO, pb + (kk >> 1) * kSliceCols + (kk & 1) * 16, sdesc_sw128(sT + kk * 32),
                         idesc, (j > 0 || kk > 0) ? 1u : 0u);
#pragma unroll
          for (int kk = 0; kk < kStream / 16; ++kk)
            umma_bf16_ts(tmem + kColO, pb + (kk >> 1) * kSliceCols + (kk & 1) * 16 + 8, sdesc_sw128(sT + kk * 32),
                         idesc, 1u);
          umma_commit(&B->buf_free[bj]);
          umma_commit(&B->empty[sj]);
          if (j == ntiles - 1) umma_commit(&B->o_full);
        }
      }
      if (*(volatile int*)&B->err && any) {
        // error: every MMA issued so far completes before TMEM is freed
        umma_commit(&B->drain);
        mbar_drain(&B->drain, 0);
      }
    }
  } else {
    // ---------------- epilogue: one fixed point per thread, column slice h ----------------
    const int t = (warp & 3) * 32 + lane;
    const int h = warp >> 2;
    const int64_t own = fixed0 + t;
    const SweepF sp = sweep_floats_of(dev, k);
    const uint64_t ahA2 = pk(sp.ahA, sp.ahA);
    float ownA;
    if (ROWS) {
      ownA = -w.rowshift[cur][own < n ? own : n - 1].x;
    } else {
      const int64_t mp = (m + 255) / 256 * 256;  // the column data are padded (offset +inf, weight 0)
      ownA = -w.colq[cur][own < mp ? own : mp - 1].x;
    }
    const uint64_t own2 = pk(ownA, ownA);
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    bool ok = true;
    for (int i = 0; i < ntiles; ++i) {
      const int b = i & 1;       // packed-pair buffer
      const int sb = i % kBufs;  // S / P buffer
      ok = mbar_wait(&B->pair_full[b], (i >> 1) & 1, B, dev);
      ok = ok && mbar_wait(&B->s_full[sb], (i / kBufs) & 1, B, dev);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const float4* pr = sPair + (size_t)b * kStream;
      const uint32_t tbase = tmem + lane_base + sb * kStream + h * kSliceCols;
      // two halves of 16 columns; P of a half replaces the S columns of that half (P_hi in
      // the first 8, P_lo in the next 8), which this thread has already read: every thread
      // writes only its own lane of its own slice, so no other thread's S is overwritten
      uint32_t vv[2][8];
      tmem_ld8(tbase, vv[0]);
      tmem_wait_ld8(vv[0]);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t phi[8], plo[8];
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int c = 2 * half + cc;
          if (c + 1 < kSliceCols / 8) tmem_ld8(tbase + (c + 1) * 8, vv[(c + 1) & 1]);
          const uint32_t(&v)[8] = vv[c & 1];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const float4 q = pr[h * kSliceCols + c * 8 + 2 * p];  // {-off pair, weight pair}
            const uint64_t z2 = pk(__uint_as_float(v[2 * p]), __uint_as_float(v[2 * p + 1]));
            const float2 vA = upk(f2fma(ahA2, z2, f2add(own2, pk(q.x, q.y))));
            const uint64_t P2 = f2mul(pk(ex2(vA.x), ex2(vA.y)), pk(q.z, q.w));
            const float2 P = upk(P2);
            const uint32_t hw = bf16x2(P.x, P.y);
            const uint64_t hf = pk(__uint_as_float(hw << 16), __uint_as_float(hw & 0xffff0000u));
            const float2 lo = upk(f2sub(P2, hf));  // exact: P - RN_bf16(P) has at most 16 significant bits
            phi[cc * 4 + p] = hw;
            plo[cc * 4 + p] = bf16x2(lo.x, lo.y);
          }
          if (c + 1 < kSliceCols / 8) tmem_wait_ld8(vv[(c + 1) & 1]);
        }
        tmem_st8(tbase + half * 16, phi);
        tmem_st8(tbase + half * 16 + 8, plo);
      }
      fence_proxy_async_smem();  // the pair buffer was read through the generic proxy
      mbar_arrive(&B->pair_empty[b]);
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&B->p_full[sb]);
    }
    // O rows of this CTA's split: coordinates [32 h, 32 h + 32) of the fixed point t
    float o[32];
    if (ntiles == 0) {
#pragma unroll
      for (int q = 0; q < 32; ++q) o[q] = 0.f;
    } else {
      ok = ok && mbar_wait(&B->o_full, 0, B, dev);
      if (!__all_sync(0xffffffffu, ok)) ok = false;
      if (ok) {
        tc_fence_after();
        tmem_ld32_wait(tmem + lane_base + kColO + h * 32, o);
      }
    }
    if (ok && own < nfixed && !*(volatile int*)&B->err) {
      float4* dst = reinterpret_cast<float4*>(part + ((int64_t)blockIdx.y * nfixed + own) * kK + h * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) dst[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// transposed bf16 copy: PT[kk][i] = Pb[i][kk] for the n_pad x 64 padded point array
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ Pb, int64_t np_pad, __nv_bfloat16* __restrict__ PT) {
  __shared__ __nv_bfloat16 tile[64][65];
  const int64_t i0 = (int64_t)blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int r = e / 64, c = e % 64;  // r: point, c: coordinate (coalesced read)
    tile[c][r] = Pb[(i0 + r) * kK + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int c = e / 64, r = e % 64;  // c: coordinate, r: point (coalesced write)
    PT[(int64_t)c * np_pad + i0 + r] = tile[c][r];
  }
}

// dx_i = 2 s (mass_i P_i - wgt_i sum_splits part_i) for rows (mass r_i, wgt q_i) and
// dy_j = 2 s (A_j P_j - w_j sum_splits part_j) for columns; coordinates q < d.
// A block of 256 threads takes kFinPoints points x 64 coordinate slots (slots q >= d idle).
// The two products are formed as float-float pairs (the rounding error of each float32
// product recovered by an fma, the mass split into float32 high and low parts) and their
// difference by TwoSum: the two terms nearly cancel where x_i is close to its barycentric
// image, and the pair keeps ~44 bits of them before the result is rounded to float32.
constexpr int kFinPoints = 4;
__global__ void __launch_bounds__(kFinPoints * 64)
k_tc_grad_fin(const float* __restrict__ part, int splits, int64_t np, int d, const float* __restrict__ P,
              const double* __restrict__ mass, const float4* __restrict__ wsrc, float s2, float* __restrict__ out) {
  __shared__ float2 msplit[kFinPoints];
  const int64_t i0 = (int64_t)blockIdx.x * kFinPoints;
  const int li = threadIdx.x >> 6;
  const int q = threadIdx.x & 63;
  const int64_t i = i0 + li;
  const bool act = i < np && q < d;
  // every load is issued before the block barrier, so that the mass loads of the first
  // threads and the partials of all threads are in flight together
  double a = 0.0;
  const bool splitter = threadIdx.x < kFinPoints && i0 + threadIdx.x < np;
  if (splitter) a = mass[i0 + threadIdx.x];
  // the splits' partials, added in split order as a float-float pair (TwoSum)
  float hi = 0.f, lo = 0.f, p = 0.f, wg = 0.f;
  if (act) {
    p = P[i * d + q];
    wg = wsrc[i].y;
    for_splits(
        splits, [&](int sp) { return part[((int64_t)sp * np + i) * kK + q]; }, [&](float v) { ff_add(hi, lo, v); });
  }
  if (threadIdx.x < kFinPoints) {
    float2 v = make_float2(0.f, 0.f);
    if (splitter) {
      const float h = (float)a;
      v = make_float2(h, (float)(a - (double)h));
    }
    msplit[threadIdx.x] = v;
  }
  __syncthreads();
  if (!act) return;
  const float2 ms = msplit[li];
  const float t1 = ms.x * p;
  const float e1 = fmaf(ms.x, p, -t1) + ms.y * p;
  const float t2 = wg * hi;
  const float e2 = fmaf(wg, hi, -t2) + wg * lo;
  float sh, se;
  two_sum(t1, -t2, sh, se);
  out[i * d + q] = s2 * (sh + (se + (e1 - e2)));
}

}  // namespace tcg

size_t tcg_smem_bytes() {
  return 1024 + (size_t)tcg::kTileBytes + 2 * (size_t)tcg::kStages * tcg::kStreamBytes + tcg::kBarBytes +
         2 * tcg::kStream * sizeof(float4);
}

cudaError_t tcg_prepare() {
  const int sm = (int)tcg_smem_bytes();
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)tcg::k_tc_grad<true>, (const void*)tcg::k_tc_grad<false>}) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  }
  return e;
}

cudaError_t tcg_transpose(const void* Pb, int64_t np_pad, void* PT, cudaStream_t st) {
  tcg::k_transpose_bf16<<<(unsigned)(np_pad / 64), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(Pb), np_pad,
                                                                   reinterpret_cast<__nv_bfloat16*>(PT));
  return cudaGetLastError();
}

int tcg_tile_fixed() { return tcg::kTile; }
int tcg_tile_stream() { return tcg::kStream; }

// one side of the gradient: rows = true (dx: fixed x, streamed y), false (dy)
cudaError_t tcg_launch(bool rows, const void* map_fixed, const void* map_stream, const void* map_streamT,
                       const Work& w, const Consts& k, int splits, float* part, cudaStream_t st) {
  const int64_t nfixed = rows ? k.n : k.m;
  const int64_t nstream = rows ? k.m : k.n;
  const int64_t ntiles = (nstream + tcg::kStream - 1) / tcg::kStream;
  const int tps = (int)((ntiles + splits - 1) / splits);
  dim3 grid((unsigned)((nfixed + tcg::kTile - 1) / tcg::kTile), (unsigned)splits);
  const CUtensorMap& mf = *reinterpret_cast<const CUtensorMap*>(map_fixed);
  const CUtensorMap& ms = *reinterpret_cast<const CUtensorMap*>(map_stream);
  const CUtensorMap& mt = *reinterpret_cast<const CUtensorMap*>(map_streamT);
  if (rows)
    tcg::k_tc_grad<true><<<grid, tcg::kThreads, tcg_smem_bytes(), st>>>(mf, ms, mt, w, k.n, k.m, tps, part, k);
  else
    tcg::k_tc_grad<false><<<grid, tcg::kThreads, tcg_smem_bytes(), st>>>(mf, ms, mt, w, k.n, k.m, tps, part, k);
  return cudaGetLastError();
}

// wsrc: the weights read after the sum, as the .y field: rows g2row (q_i), columns the
// state's colq (w_j), chosen by the caller with the state's buffer parity
cudaError_t tcg_finalize(bool rows, const float* part, int splits, const Work& w, const Consts& k, const float* P,
                         const double* r, const float4* wsrc, float* out, cudaStream_t st) {
  const int64_t np = rows ? k.n : k.m;
  const unsigned blocks = (unsigned)((np + tcg::kFinPoints - 1) / tcg::kFinPoints);
  tcg::k_tc_grad_fin<<<blocks, tcg::kFinPoints * 64, 0, st>>>(part, splits, np, (int)k.d, P, rows ? r : w.colA,
                                                              wsrc, (float)(2.0 * k.s), out);
  return cudaGetLastError();
}

}  // namespace lamp
