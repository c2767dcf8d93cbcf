// tcgen05 (5th-generation tensor core) sweeps of the LAMP hot path for the
// squared-Euclidean cost in dot form, BF16 points, FP32 accumulation in TMEM.
//
// The row sweep G1 keeps a 256-row x tile fixed (two 128-row halves) and streams
// 64-row y tiles: per streamed tile two MMAs D_a = Xb[half a, 0:64] * Yb[tile, 0:64]^T
// (M = 128, N = 64, K = 64).  The column sweep G2 does the same with the roles of x and
// y exchanged (y tile fixed, x tiles streamed).  Operands are K-major bf16 tiles staged
// by TMA with 128-byte swizzle.  With bf16 operands every product is exact in fp32 and
// the MMA's accumulation does not depend on which operand is A: D'[j][i] and D[i][j]
// are bit-identical, so the column sweep's exponents equal the row sweep's and its
// normalisation matches the row sums exactly.
//
// CTA = 10 warps: warps 0-7 read TMEM and run the exponent / ex2 / accumulation
// epilogue with packed f32x2 arithmetic over pairs of entries; warp w owns TMEM lanes
// 32 (w % 4) .. + 31 of both accumulator halves, i.e. two rows of D per thread (G1: rows
// t and 128 + t of the fixed tile; G2: two columns of X), and columns
// [32 (w / 4), + 32) of each streamed tile.  Each thread thus reads every column's
// packed offsets / weights once for two rows: the broadcast shared-memory loads of
// those data, not the ex2 or the FMA pipe, bounded a one-row-per-thread epilogue.
// Warp 8 issues TMA loads, warp 9 issues tcgen05.mma.  Two TMEM buffers (2 x 128
// columns: two 64-column halves each) let the MMAs of tile i+1 overlap the epilogue of
// tile i; a 4-stage shared-memory ring feeds the streamed operand.
//
// Every mbarrier wait is bounded: on timeout the kernel records LAMP_E_TIMEOUT in
// the device status word, stops issuing work, waits (bounded) for its own copies
// and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "lamp_async.cuh"
#include "lamp_common.cuh"
#include "lamp_tc.cuh"

namespace lamp {

namespace tc {

constexpr int kTile = 128;       // rows of a fixed half tile = MMA M; padding unit of the bf16 copies
constexpr int kFixed = 2 * kTile;  // rows of the fixed tile (two MMA halves)
constexpr int kStream = 64;      // rows of a streamed tile = MMA N
constexpr int kK = 64;           // K extent (points zero-padded to 64 coordinates)
constexpr int kStages = 4;       // streamed-operand ring
constexpr int kTileBytes = kTile * kK * 2;      // 16 KiB per 128-row bf16 half tile
constexpr int kStreamBytes = kStream * kK * 2;  // 8 KiB per streamed bf16 tile
constexpr int kEpiWarps = 8;      // kSlices warps per TMEM lane quadrant, one column slice each
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kSlices = kEpiWarps / 4;            // column slices of a streamed tile
constexpr int kSliceCols = kStream / kSlices;     // columns per slice (multiple of 16)
static_assert(kEpiWarps % 4 == 0 && kStream % kSlices == 0 && kSliceCols % 8 == 0, "epilogue layout");
// padding unit of the bf16 copies and of the per-point data arrays: whole fixed halves and
// whole streamed tiles, lcm(kTile, kStream)
constexpr int64_t gcd_c(int64_t a, int64_t b) { return b == 0 ? a : gcd_c(b, a % b); }
constexpr int64_t kPad = kTile / gcd_c(kTile, kStream) * kStream;
constexpr int kProducerWarp = kEpiWarps;
constexpr int kMmaWarp = kEpiWarps + 1;
constexpr int kThreads = (kEpiWarps + 2) * 32;
constexpr uint32_t kTmemCols = 256;         // two buffers x two 64-column FP32 accumulators
constexpr uint32_t kWaitLimit = async::kWaitLimit;  // bounded spin on every mbarrier
constexpr int kTimeoutStatus = async::kTimeoutStatus;

struct __align__(8) Bars {
  uint64_t fixed_full;
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t tmem_full[2];
  uint64_t tmem_empty[2];
  uint64_t pair_full[2];   // packed offsets / weights of the streamed tile landed (bulk copy)
  uint64_t pair_empty[2];  // epilogue finished reading them
  uint32_t tmem_base;
  int err;
};
constexpr int kBarBytes = 256;
static_assert(sizeof(Bars) <= kBarBytes, "barrier block");

using async::bulk_load;
using async::fence_proxy_async_smem;
using async::mbar_arrive;
using async::mbar_drain;
using async::mbar_expect_tx;
using async::mbar_init;
using async::smem_u32;
using async::tma_load_2d;

// bounded wait on one of this CTA's barriers (error flag in the barrier block)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, Bars* B, DevState* dev,
                                          uint32_t limit = async::kWaitLimit) {
  return async::mbar_wait(bar, parity, &B->err, dev, limit);
}

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes at two addresses (the two
// accumulator halves), without waiting: tcgen05.ld writes its destination registers
// asynchronously, until tcgen05.wait::ld.
__device__ __forceinline__ void tmem_ld8x2(uint32_t ta, uint32_t tb, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(ta), "r"(tb)
      : "memory");
}

// wait for this thread's TMEM loads; the registers they write are in-out operands, so
// the compiler orders every use (and any copy) of them after the wait
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                 "+r"(v[15])
               :
               : "memory");
}



// barrier over the epilogue threads (named barrier 1) returning the OR of `v`
// across them, so that every epilogue warp takes the same branch
__device__ __forceinline__ bool epi_bar_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n"
      ".reg .pred p, q;\n"
      "setp.ne.u32 p, %1, 0;\n"
      "bar.red.or.pred q, 1, %2, p;\n"
      "selp.u32 %0, 1, 0, q;\n"
      "}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kEpiThreads)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

// ROWS = true: G1 (fixed x tile, streamed y tiles, per-row sums of both streams)
// ROWS = false: G2 (fixed y tile, streamed x tiles, per-column sums of both streams)
// WC: column sweep of an evaluation pass (also accumulates sum_i z_ij X_ij for <C, X^t>)
// map_fixed: 128-row boxes of the fixed operand; map_stream: 64-row boxes of the streamed one
// MODE (row sweeps only): kSums, the iteration's sums; kMax, the row maxima of stream A's
// exponent without row shift, a z_ij - Bq_j (the prime pass that sets the row shifts);
// kMax2, the refined row maxima u_ij = a z_ij - (Rq_i + Bq_j) - Br_j with the multiplier's
// low part (the eta = 0 dual bound's second pass); kKmax, the row maxima of D_ij and of
// -D_ij, D_ij = |x_i|^2 + |y_j|^2 - 2 x_i.y_j (the K pass: the row data hold |x_i|^2, the
// pair data -offA = |y_j|^2, columns past m are skipped).  The maxima go to rowmax per split.
constexpr int kSums = 0, kMax = 1, kMax2 = 2, kKmax = 3;
template <bool ROWS, int WC, int MODE = kSums>
__global__ void __launch_bounds__(kThreads, 2)
k_tc_sweep(const __grid_constant__ CUtensorMap map_fixed, const __grid_constant__ CUtensorMap map_stream,
           const Work w, int64_t n, int64_t m, int tiles_per_split, const Consts k) {
  DevState* __restrict__ dev = w.dev;
  if (dev->done) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sFixed = smem;                         // two 16 KiB halves
  unsigned char* sStream = smem + 2 * kTileBytes;       // kStages x 8 KiB
  Bars* B = reinterpret_cast<Bars*>(sStream + kStreamBytes * kStages);
  // per streamed tile, double-buffered: the packed-pair data of its 64 entries (32 pairs,
  // two float4 each; G1: column offsets / weights, G2: row offsets / weights), copied by
  // a bulk copy from the packed-pair arrays the finalize kernels write
  float4* sPair = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(B) + kBarBytes);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int cur = dev->cur;
  const int64_t fixed0 = (int64_t)blockIdx.x * kFixed;  // first row (G1) / column (G2) of the fixed tile
  const int64_t nstream = ROWS ? m : n;
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
    for (int b = 0; b < 2; ++b) {
      mbar_init(&B->tmem_full[b], 1);
      mbar_init(&B->tmem_empty[b], kEpiThreads);
      mbar_init(&B->pair_full[b], 1);
      mbar_init(&B->pair_empty[b], kEpiThreads);
    }
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
    if (lane == 0) {
      const float4* __restrict__ pair_src = ROWS ? w.colq2[cur] : w.g2row2;
      int issued = 0, pissued = 0;
      // the fixed tile: two 128-row boxes (rows beyond the padded array read as zeros)
      mbar_expect_tx(&B->fixed_full, 2 * kTileBytes);
      tma_load_2d(sFixed, &map_fixed, &B->fixed_full, 0, (int)fixed0);
      tma_load_2d(sFixed + kTileBytes, &map_fixed, &B->fixed_full, 0, (int)(fixed0 + kTile));
      for (int i = 0; i < ntiles; ++i) {
        const int s = i % kStages;
        const int b = i & 1;
        if (i >= kStages && !mbar_wait(&B->empty[s], ((i / kStages) & 1) ^ 1, B, dev)) break;
        mbar_expect_tx(&B->full[s], kStreamBytes);
        tma_load_2d(sStream + s * kStreamBytes, &map_stream, &B->full[s], 0, (int)((it0 + i) * kStream));
        issued = i + 1;
        if (i >= 2 && !mbar_wait(&B->pair_empty[b], ((i >> 1) - 1) & 1, B, dev)) break;
        mbar_expect_tx(&B->pair_full[b], kStream * sizeof(float4));
        bulk_load(sPair + (size_t)b * kStream, pair_src + (it0 + i) * kStream, kStream * sizeof(float4),
                  &B->pair_full[b]);
        pissued = i + 1;
      }
      if (*(volatile int*)&B->err) {
        // error: let this thread's copies in flight land before the CTA exits
        mbar_drain(&B->fixed_full, 0);
        for (int i = issued - kStages < 0 ? 0 : issued - kStages; i < issued; ++i)
          mbar_drain(&B->full[i % kStages], (i / kStages) & 1);
        for (int i = pissued - 2 < 0 ? 0 : pissued - 2; i < pissued; ++i) mbar_drain(&B->pair_full[i & 1], (i >> 1) & 1);
      }
    }
  } else if (warp == kMmaWarp) {
    // ------ MMA issuer: D[buffer][half a] = A(fixed half a) * B(streamed)^T, a = 0, 1 ------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kTile, kStream);
      int issued = 0;
      if (mbar_wait(&B->fixed_full, 0, B, dev)) {
        const uint32_t sF = smem_u32(sFixed);
        const uint32_t sS = smem_u32(sStream);
        for (int i = 0; i < ntiles; ++i) {
          const int s = i % kStages;
          const int b = i & 1;
          if (!mbar_wait(&B->full[s], (i / kStages) & 1, B, dev)) break;
          if (i >= 2 && !mbar_wait(&B->tmem_empty[b], ((i >> 1) - 1) & 1, B, dev)) break;
          tc_fence_after();
          const uint32_t bBase = sS + s * kStreamBytes;
#pragma unroll
          for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int kk = 0; kk < kK / 16; ++kk)
              umma_bf16(tmem + b * (2 * kStream) + a * kStream, sdesc_sw128(sF + a * kTileBytes + kk * 32),
                        sdesc_sw128(bBase + kk * 32), idesc, kk > 0);
          umma_commit(&B->empty[s]);
          umma_commit(&B->tmem_full[b]);
          issued = i + 1;
        }
      }
      if (*(volatile int*)&B->err) {
        // error: wait for the MMAs already issued before TMEM is freed
        for (int i = issued - 2 < 0 ? 0 : issued - 2; i < issued; ++i) mbar_drain(&B->tmem_full[i & 1], (i >> 1) & 1);
      }
    }
  } else {
    // ---- epilogue: warps 0 .. kEpiWarps-1; TMEM lane t of both halves, column slice h ----
    const int t = (warp & 3) * 32 + lane;  // TMEM lane (0..127); rows t and 128 + t of the fixed tile
    const int h = warp >> 2;               // columns [h kSliceCols, (h + 1) kSliceCols) of each streamed tile
    const SweepF sp = sweep_floats_of(dev, k);
    // v^A = a^A z + own + off with a^A rounded to float32 (ah): dropping the low part al
    // changes v by at most half an ulp of a^A z, the order of the rounding of z itself in
    // the MMA's FP32 accumulation (the float32 CUDA-core paths keep al)
    const uint64_t ahA2 = MODE == kKmax ? pk(-2.f, -2.f) : pk(sp.ahA, sp.ahA);
    const uint64_t alA2 = pk(sp.alA, sp.alA);  // kMax2 only
    const float dal = sp.dal;  // stream B: v^B = (a^B - a^A) z + (v^A + dB)
    const uint64_t da2 = pk(dal, dal);
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;  // TMEM lane field
    // the own offsets of this thread's two fixed points (G1: the rows' shifts; G2: the
    // columns' offsets, negated, and their dB as stored in the pair arrays); points past
    // the end read a clamped (G1) or padding (G2) entry and are never written
    uint64_t ownA2[2], ownD2[2] = {0ull, 0ull};
    int64_t own[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      own[r] = fixed0 + r * kTile + t;
      if (ROWS) {
        const float2 rq = w.rowshift[cur][own[r] < n ? own[r] : n - 1];
        // the prime pass has no row shift yet; the K pass reads |x_i|^2
        const float o = MODE == kMax ? 0.f : (MODE == kKmax ? rq.x : -rq.x);
        ownA2[r] = pk(o, o);
      } else {
        const int64_t mp = (m + kPad - 1) / kPad * kPad;  // the column data are padded to mp
        const int64_t oc = own[r] < mp ? own[r] : mp - 1;
        const float4 cq = w.colq[cur][oc];  // padded columns: {+inf, 0, +inf, 0}
        ownA2[r] = pk(-cq.x, -cq.x);
        const float db = pair_dB(w.colq2[cur], oc);  // padding: -2^100
        ownD2[r] = pk(db, db);
      }
    }
    float hiA[2] = {0.f, 0.f}, loA[2] = {0.f, 0.f}, hiB[2] = {0.f, 0.f}, loB[2] = {0.f, 0.f};
    float hiC[2] = {0.f, 0.f}, loC[2] = {0.f, 0.f};
    float mxA[2] = {-INFINITY, -INFINITY};  // kMax, kMax2, kKmax: running row maxima
    float mnA[2] = {-INFINITY, -INFINITY};  // kKmax: running row maxima of -D
    // packed pair sums of this thread's two points over one streamed tile
    uint64_t accA[2], accB[2], accC[2];
    uint32_t vv[2][16];  // two TMEM chunks: the one evaluated and the one in flight
    constexpr int kChunks = kSliceCols / 8;
    for (int i = 0; i < ntiles; ++i) {
      const int b = i & 1;
      bool ok = mbar_wait(&B->pair_full[b], (i >> 1) & 1, B, dev);
      ok = ok && mbar_wait(&B->tmem_full[b], (i >> 1) & 1, B, dev);
      // warp-uniform decision before the .sync.aligned TMEM loads
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const float4* pr = sPair + (size_t)b * kStream;
      const uint32_t tbase = tmem + lane_base + b * (2 * kStream) + h * kSliceCols;
#pragma unroll
      for (int r = 0; r < 2; ++r) accA[r] = accB[r] = accC[r] = 0ull;
      // chunks of 8 columns of both halves, software-pipelined: the loads of chunk c + 1
      // are in flight while chunk c is evaluated (v[0..7] row / column t, v[8..15] row /
      // column 128 + t)
      tmem_ld8x2(tbase, tbase + kStream, vv[0]);
      tmem_wait_ld(vv[0]);
#pragma unroll
      for (int c = 0; c < kChunks; ++c) {
        if (c + 1 < kChunks) tmem_ld8x2(tbase + (c + 1) * 8, tbase + kStream + (c + 1) * 8, vv[(c + 1) & 1]);
        const uint32_t(&v)[16] = vv[c & 1];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int col = h * kSliceCols + c * 8 + 2 * p;  // first column of the pair in the tile
          const float4 qa = pr[col];
          if constexpr (MODE != kSums) {
            // {-Bq pair, Br pair} (kMax2) or {-Bq pair, weights} (kMax): no exponentials
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              const uint64_t z2 = pk(__uint_as_float(v[8 * r + 2 * p]), __uint_as_float(v[8 * r + 2 * p + 1]));
              uint64_t u = f2fma(ahA2, z2, f2add(ownA2[r], pk(qa.x, qa.y)));
              if constexpr (MODE == kMax2) u = f2sub(f2fma(alA2, z2, u), pk(qa.z, qa.w));
              const float2 uf = upk(u);
              if constexpr (MODE == kKmax) {
                const int64_t gcol = (it0 + i) * kStream + col;  // padding columns hold no point
                const float d0 = gcol < m ? uf.x : -INFINITY, d1 = gcol + 1 < m ? uf.y : -INFINITY;
                const float e0 = gcol < m ? -uf.x : -INFINITY, e1 = gcol + 1 < m ? -uf.y : -INFINITY;
                mxA[r] = fmaxf(mxA[r], fmaxf(d0, d1));
                mnA[r] = fmaxf(mnA[r], fmaxf(e0, e1));
                continue;
              }
              mxA[r] = fmaxf(mxA[r], fmaxf(uf.x, uf.y));
            }
            continue;
          }
          const float4 qb = pr[col + 1];
          const uint64_t offA2 = pk(qa.x, qa.y), wA2 = pk(qa.z, qa.w);
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const uint64_t z2 = pk(__uint_as_float(v[8 * r + 2 * p]), __uint_as_float(v[8 * r + 2 * p + 1]));
            const uint64_t vA = f2fma(ahA2, z2, f2add(ownA2[r], offA2));
            // G1: the inner column's dB from the pair data; G2: the own column's
            const uint64_t vB = f2fma(da2, z2, f2add(vA, ROWS ? pk(qb.x, qb.y) : ownD2[r]));
            const float2 vAf = upk(vA), vBf = upk(vB);
            const uint64_t eA = pk(ex2(vAf.x), ex2(vAf.y));
            const uint64_t eB = pk(ex2(vBf.x), ex2(vBf.y));
            if (WC) {
              const uint64_t pA = f2mul(eA, wA2);
              accA[r] = f2add(accA[r], pA);
              accC[r] = f2fma(z2, pA, accC[r]);
            } else {
              accA[r] = f2fma(eA, wA2, accA[r]);
            }
            // G1: stream B's column weight is inside dB; G2: weight by the row's q^B
            if (ROWS) accB[r] = f2add(accB[r], eB);
            else accB[r] = f2fma(eB, pk(qb.z, qb.w), accB[r]);
          }
        }
        if (c + 1 < kChunks) tmem_wait_ld(vv[(c + 1) & 1]);
      }
#pragma unroll
      for (int r = 0; r < 2 && MODE == kSums; ++r) {
        const float2 a2 = upk(accA[r]), b2 = upk(accB[r]);
        ff_add(hiA[r], loA[r], a2.x + a2.y);
        ff_add(hiB[r], loB[r], b2.x + b2.y);
        if (WC) {
          const float2 c2 = upk(accC[r]);
          ff_add(hiC[r], loC[r], c2.x + c2.y);
        }
      }
      tc_fence_before();
      mbar_arrive(&B->tmem_empty[b]);
      // the pair buffer was read through the generic proxy and the producer's next bulk
      // copy into it is an async-proxy write: without the proxy fence that write can
      // overtake these reads (a write-after-read race across proxies)
      fence_proxy_async_smem();
      mbar_arrive(&B->pair_empty[b]);
    }
    // combine the column slices h of each point in a buffer of its own (generic proxy only)
    double* comb = reinterpret_cast<double*>(sPair + 2 * kStream);
    if (h >= 1) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        double* cb = comb + ((size_t)(h - 1) * kFixed + r * kTile + t) * 3;
        if constexpr (MODE != kSums) {
          cb[0] = (double)mxA[r];
          cb[1] = (double)mnA[r];
          continue;
        }
        cb[0] = (double)hiA[r] + (double)loA[r];
        cb[1] = (double)hiB[r] + (double)loB[r];
        cb[2] = (double)hiC[r] + (double)loC[r];
      }
    }
    epi_bar();
    if (MODE != kSums && h == 0 && !*(volatile int*)&B->err) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float mx = mxA[r], mn = mnA[r];
        for (int hh = 1; hh < kSlices; ++hh) {
          mx = fmaxf(mx, (float)comb[((size_t)(hh - 1) * kFixed + r * kTile + t) * 3]);
          mn = fmaxf(mn, (float)comb[((size_t)(hh - 1) * kFixed + r * kTile + t) * 3 + 1]);
        }
        if (own[r] < n) {
          // the K pass: max D and max -D; otherwise stream B's maxima are not used under the
          // shared row shift (the B shift is A's)
          w.rowmax[((int64_t)blockIdx.y * 2 + 0) * n + own[r]] = mx;
          w.rowmax[((int64_t)blockIdx.y * 2 + 1) * n + own[r]] = MODE == kKmax ? mn : mx;
        }
      }
    }
    if (MODE == kSums && h == 0 && !*(volatile int*)&B->err) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        double sA = (double)hiA[r] + (double)loA[r];
        double sB = (double)hiB[r] + (double)loB[r];
        double sC = (double)hiC[r] + (double)loC[r];
        for (int hh = 1; hh < kSlices; ++hh) {
          const double* cb = comb + ((size_t)(hh - 1) * kFixed + r * kTile + t) * 3;
          sA += cb[0];
          sB += cb[1];
          sC += cb[2];
        }
        if (ROWS) {
          if (own[r] < n) {
            w.rowpart[((int64_t)blockIdx.y * 2 + 0) * n + own[r]] = sA;
            w.rowpart[((int64_t)blockIdx.y * 2 + 1) * n + own[r]] = sB;
          }
        } else if (own[r] < m) {
          constexpr int na = WC ? 3 : 2;  // the layout k_col_fin reads for this pass
          w.colpart[((int64_t)blockIdx.y * na + 0) * m + own[r]] = sA;
          w.colpart[((int64_t)blockIdx.y * na + 1) * m + own[r]] = sB;
          if (WC) w.colpart[((int64_t)blockIdx.y * na + 2) * m + own[r]] = sC;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// x (n x d float32) -> rounded float32 copy (n x d) and bf16 copy (n_pad x 64, zero padded)
__global__ void k_to_bf16(const float* __restrict__ P, int64_t np, int64_t np_pad, int d, float* __restrict__ Pr,
                          __nv_bfloat16* __restrict__ Pb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np_pad * kK) return;
  const int64_t i = e / kK;
  const int kk = (int)(e - i * kK);
  float v = 0.f;
  if (i < np && kk < d) v = P[i * d + kk];
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  Pb[e] = b;
  if (i < np && kk < d) Pr[i * d + kk] = __bfloat162float(b);
}

__global__ void k_fill_pad4(float4* __restrict__ a, int64_t from, int64_t to) {
  const int64_t i = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < to) a[i] = make_float4(INFINITY, 0.f, INFINITY, 0.f);
}

// packed-pair arrays: every half starts as padding {-off = -2^100, wgt = 0}
__global__ void k_fill_pairs(float4* __restrict__ a, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // padding: a finite offset far below any real one (differences of two padding offsets,
  // which the direct-form sweeps take, stay 0 instead of inf - inf), zero weight
  if (i < count) a[i] = make_float4(-0x1p100f, -0x1p100f, 0.f, 0.f);
}

// Self-test of the bounded wait: one thread waits on a barrier that nothing arrives on
// (phase 0 of a fresh barrier with one expected arrival); after `limit` polls the wait
// gives up, records LAMP_E_TIMEOUT in dev->status and the kernel returns normally.
__global__ void k_wait_selftest(uint32_t limit, DevState* dev) {
  __shared__ __align__(8) Bars B;
  if (threadIdx.x == 0) {
    mbar_init(&B.full[0], 1);
    B.err = 0;
    async::mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = mbar_wait(&B.full[0], 0, &B, dev, limit);
    if (ok) atomicExch(&dev->status, -1);  // impossible: nothing arrives
  }
}

}  // namespace tc

int tc_wait_selftest(uint32_t polls, int* status) {
  DevState* d = nullptr;
  if (cudaMalloc(&d, sizeof(DevState)) != cudaSuccess) return 3;
  cudaError_t e = cudaMemset(d, 0, sizeof(DevState));
  if (e == cudaSuccess) {
    tc::k_wait_selftest<<<1, 32>>>(polls, d);
    e = cudaGetLastError();
  }
  DevState h{};
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(DevState), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return 2;
  *status = h.status;
  return 0;
}

size_t tc_smem_bytes() {
  // alignment slack + fixed tile (two halves) + ring + barriers + packed pairs (2 x 64 float4)
  // + the epilogue's combine buffer ((slices - 1) x 256 points x 3 doubles)
  return 1024 + (size_t)tc::kTileBytes * 2 + (size_t)tc::kStreamBytes * tc::kStages + tc::kBarBytes +
         2 * tc::kStream * sizeof(float4) + (size_t)(tc::kSlices - 1) * tc::kFixed * 3 * sizeof(double);
}

int64_t tc_pad(int64_t v) { return (v + tc::kPad - 1) / tc::kPad * tc::kPad; }

cudaError_t tc_convert(const float* P, int64_t np, int d, float* Pr, void* Pb, cudaStream_t st) {
  const int64_t np_pad = tc_pad(np);
  const int64_t total = np_pad * tc::kK;
  tc::k_to_bf16<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, np, np_pad, d, Pr,
                                                                   reinterpret_cast<__nv_bfloat16*>(Pb));
  return cudaGetLastError();
}

cudaError_t tc_fill_pads(float4* a, int64_t from, int64_t to, cudaStream_t st) {
  if (to <= from) return cudaSuccess;
  tc::k_fill_pad4<<<(unsigned)((to - from + 255) / 256), 256, 0, st>>>(a, from, to);
  return cudaGetLastError();
}

cudaError_t tc_fill_pairs(float4* a, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  tc::k_fill_pairs<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(a, count);
  return cudaGetLastError();
}

// encode a 2-D bf16 tensor map over a (rows_pad x 64) row-major array, box_rows x 64 boxes,
// 128B swizzle (box_rows: 128 for the fixed halves, 64 for the streamed tiles)
cudaError_t tc_make_map(void* map_out, const void* base, int64_t rows_pad, int box_rows) {
  return tc_make_map2(map_out, base, tc::kK, rows_pad, tc::kK, box_rows);
}

cudaError_t tc_make_map2(void* map_out, const void* base, int64_t inner, int64_t rows, int box_inner, int box_rows) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<EncodeFn>(p);
  }
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_prepare() {
  const int sm = (int)tc_smem_bytes();
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)tc::k_tc_sweep<true, 0>, (const void*)tc::k_tc_sweep<false, 0>,
                        (const void*)tc::k_tc_sweep<false, 1>, (const void*)tc::k_tc_sweep<true, 0, tc::kMax>,
                        (const void*)tc::k_tc_sweep<true, 0, tc::kMax2>,
                        (const void*)tc::k_tc_sweep<true, 0, tc::kKmax>}) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    // prefer the largest shared-memory carveout: two CTAs per SM need 2 x ~75 KB
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  }
  return e;
}

int tc_blocks_per_sm(int which) {
  // resident CTAs per SM from the kernel's registers, its shared memory and TMEM (two
  // 256-column allocations fill the 512 columns of an SM); the occupancy API assumes the
  // default shared-memory carveout and undercounts, while the sweeps run at the maximum
  cudaFuncAttributes fa{};
  cudaError_t e = which == 0 ? cudaFuncGetAttributes(&fa, tc::k_tc_sweep<true, 0>)
                             : cudaFuncGetAttributes(&fa, tc::k_tc_sweep<false, 1>);
  int dev = 0, smem_sm = 0, regs_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e != cudaSuccess || fa.numRegs <= 0) return 1;
  const int by_regs = regs_sm / (fa.numRegs * tc::kThreads);
  const int by_smem = smem_sm / (int)(tc_smem_bytes() + fa.sharedSizeBytes + 1024);
  int nb = by_regs < by_smem ? by_regs : by_smem;
  if (nb > 2) nb = 2;
  return nb > 0 ? nb : 1;
}

int tc_tile_fixed() { return tc::kFixed; }
int tc_tile_stream() { return tc::kStream; }

cudaError_t tc_launch_sweep(bool rows, int eval, const Geometry& g, const Work& w, const Consts& k, int splits,
                            cudaStream_t st) {
  const int64_t nfixed = rows ? k.n : k.m;
  const int64_t nstream = rows ? k.m : k.n;
  const int64_t ntiles = (nstream + tc::kStream - 1) / tc::kStream;
  const int tps = (int)((ntiles + splits - 1) / splits);
  dim3 grid((unsigned)((nfixed + tc::kFixed - 1) / tc::kFixed), (unsigned)splits);
  // G1: x fixed (128-row boxes), y streamed (64-row boxes); G2: the reverse
  const CUtensorMap& mf = *reinterpret_cast<const CUtensorMap*>(rows ? g.map_x : g.map_y);
  const CUtensorMap& ms = *reinterpret_cast<const CUtensorMap*>(rows ? g.map_y64 : g.map_x64);
  if (rows)
    tc::k_tc_sweep<true, 0><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mf, ms, w, k.n, k.m, tps, k);
  else if (eval)
    tc::k_tc_sweep<false, 1><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mf, ms, w, k.n, k.m, tps, k);
  else
    tc::k_tc_sweep<false, 0><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mf, ms, w, k.n, k.m, tps, k);
  return cudaGetLastError();
}

// row maxima on the tensor cores: mode 1 = the prime pass (a z - Bq, no row shift), mode 2 =
// the refined pass (a z - (Rq + Bq) - Br), mode 3 = the K pass (max D and max -D); per split
// into w.rowmax, as the row sweep's grid
cudaError_t tc_launch_rowmax(int mode, const Geometry& g, const Work& w, const Consts& k, int splits, cudaStream_t st) {
  const int64_t ntiles = (k.m + tc::kStream - 1) / tc::kStream;
  const int tps = (int)((ntiles + splits - 1) / splits);
  dim3 grid((unsigned)((k.n + tc::kFixed - 1) / tc::kFixed), (unsigned)splits);
  const CUtensorMap& mf = *reinterpret_cast<const CUtensorMap*>(g.map_x);
  const CUtensorMap& ms = *reinterpret_cast<const CUtensorMap*>(g.map_y64);
  if (mode == 1)
    tc::k_tc_sweep<true, 0, tc::kMax><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mf, ms, w, k.n, k.m, tps, k);
  else if (mode == 2)
    tc::k_tc_sweep<true, 0, tc::kMax2><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mf, ms, w, k.n, k.m, tps, k);
  else
    tc::k_tc_sweep<true, 0, tc::kKmax><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mf, ms, w, k.n, k.m, tps, k);
  return cudaGetLastError();
}

}  // namespace lamp
