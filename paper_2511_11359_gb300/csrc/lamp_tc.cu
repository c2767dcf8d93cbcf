// tcgen05 (5th-generation tensor core) sweeps of the LAMP hot path for the
// squared-Euclidean cost in dot form, BF16 points, FP32 accumulation in TMEM.
//
// The row sweep G1 computes, per 128-row x tile (fixed) and 128-column y tile
// (streamed), D = Xb[rows, 0:64] * Yb[cols, 0:64]^T; the column sweep G2 computes
// D' = Yb[cols] * Xb[rows]^T with the y tile fixed and x tiles streamed (A and B
// are 128 x 64 K-major bf16 tiles staged by TMA with 128-byte swizzle).  With
// bf16 operands every product is exact in fp32 and the MMA's accumulation does
// not depend on which operand is A: D'[j][i] and D[i][j] are bit-identical, so
// the column sweep's exponents equal the row sweep's and its normalisation
// matches the row sums exactly.  In both sweeps one thread owns one TMEM lane
// (a row of D in G1, a column of X in G2) and accumulates in registers.
//
// CTA = 10 warps: warps 0-7 read TMEM (warp w owns lanes 32(w%4).. and columns
// [64 (w/4), 64 (w/4) + 64) of each 128-column accumulator) and run the exponent /
// ex2 / accumulation epilogue with packed f32x2 arithmetic over pairs of entries;
// warp 8 issues TMA loads, warp 9 issues tcgen05.mma.  Two TMEM accumulators (2 x 128 columns)
// let the MMA of tile i+1 overlap the epilogue of tile i; a 4-stage shared-memory
// ring feeds the streamed operand.
//
// Every mbarrier wait is bounded: on timeout the kernel records LAMP_E_TIMEOUT in
// the device status word, stops issuing work, waits (bounded) for its own copies
// and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "lamp_common.cuh"

namespace lamp {

namespace tc {

constexpr int kTile = 128;       // rows per A tile = columns per B tile = MMA M = N
constexpr int kK = 64;           // K extent (points zero-padded to 64 coordinates)
constexpr int kStages = 4;       // streamed-operand ring
constexpr int kTileBytes = kTile * kK * 2;  // 16 KiB per bf16 tile
constexpr int kEpiWarps = 8;      // two warps per TMEM lane quadrant, each takes half the columns
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kProducerWarp = kEpiWarps;
constexpr int kMmaWarp = kEpiWarps + 1;
constexpr int kThreads = (kEpiWarps + 2) * 32;
constexpr uint32_t kTmemCols = 256;         // two 128-column FP32 accumulators
constexpr uint32_t kWaitLimit = 1u << 24;   // bounded spin on every mbarrier
constexpr int kTimeoutStatus = 6;           // LAMP_E_TIMEOUT

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

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false when the CTA is in error or the limit ran out (then the error is recorded)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, Bars* B, DevState* dev,
                                          uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*(volatile int*)&B->err) return false;
  }
  atomicExch(&B->err, 1);
  atomicExch(&dev->status, kTimeoutStatus);
  return false;
}

// drain wait used on the error path: only the iteration limit, no early exit
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// plain (untiled) bulk copy global -> shared, completion counted on an mbarrier;
// both addresses 16-byte aligned, size a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (bf16 in, fp32 accumulate)
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}


// 32 consecutive FP32 columns of this warp's 32 TMEM lanes, load and wait in ONE asm
// statement: the destination registers of tcgen05.ld are written asynchronously until
// tcgen05.wait::ld, and if the two were separate statements the compiler could copy
// or spill those registers in between (it believes they are already final).
__device__ __forceinline__ void tmem_ld32_wait(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
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

// Shared-memory matrix descriptor of a K-major bf16 tile written by TMA with
// 128-byte swizzle: rows of 128 bytes, 8-row (1024-byte) swizzle atoms, so the
// stride between 8-row groups is 1024 bytes; the leading offset is unused for
// this layout; bits 46-47 hold the descriptor version 1; layout type 2 = 128B
// swizzle.  Stepping K by 16 elements advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D fp32, A and B bf16, both K-major, M = N = 128.
__host__ __device__ constexpr uint32_t idesc_bf16_128x128() {
  return (1u << 4)                      // D format: f32
         | (1u << 7)                    // A format: bf16
         | (1u << 10)                   // B format: bf16
         | ((uint32_t)(kTile >> 3) << 17)  // N >> 3
         | ((uint32_t)(kTile >> 4) << 24); // M >> 4
}

// ROWS = true: G1 (fixed x tile, streamed y tiles, per-row sums of both streams)
// ROWS = false: G2 (fixed y tile, streamed x tiles, per-column sums of both streams
// and of z X for <C, X>)
// WC: column sweep of an evaluation pass (also accumulates sum_i z_ij X_ij for <C, X^t>)
template <bool ROWS, int WC>
__global__ void __launch_bounds__(kThreads, 2)
k_tc_sweep(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_y, const Work w,
           int64_t n, int64_t m, int tiles_per_split, const Consts k) {
  DevState* __restrict__ dev = w.dev;
  if (dev->done) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sFixed = smem;
  unsigned char* sStream = smem + kTileBytes;
  Bars* B = reinterpret_cast<Bars*>(smem + kTileBytes * (1 + kStages));
  // per streamed tile, double-buffered: for each pair of entries p, two float4
  //   [2p] = {-offA_2p, -offA_2p+1, wgtA_2p, wgtA_2p+1}, [2p+1] = the same for stream B
  // (G1: column offsets / weights w_j; G2: row offsets / weights q_i), copied by TMA
  // from the packed-pair arrays the finalize kernels write
  float4* sPair = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(B) + kBarBytes);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int cur = dev->cur;
  const int64_t fixed0 = (int64_t)blockIdx.x * kTile;  // first row (G1) / column (G2) of the fixed tile
  const int64_t nstream = ROWS ? m : n;
  const int64_t ntiles_all = (nstream + kTile - 1) / kTile;
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
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
      mbar_expect_tx(&B->fixed_full, kTileBytes);
      tma_load_2d(sFixed, ROWS ? &map_x : &map_y, &B->fixed_full, 0, (int)fixed0);
      for (int i = 0; i < ntiles; ++i) {
        const int s = i % kStages;
        const int b = i & 1;
        if (i >= kStages && !mbar_wait(&B->empty[s], ((i / kStages) & 1) ^ 1, B, dev)) break;
        mbar_expect_tx(&B->full[s], kTileBytes);
        tma_load_2d(sStream + s * kTileBytes, ROWS ? &map_y : &map_x, &B->full[s], 0, (int)((it0 + i) * kTile));
        issued = i + 1;
        if (i >= 2 && !mbar_wait(&B->pair_empty[b], ((i >> 1) - 1) & 1, B, dev)) break;
        mbar_expect_tx(&B->pair_full[b], kTile * sizeof(float4));
        bulk_load(sPair + (size_t)b * kTile, pair_src + (it0 + i) * kTile, kTile * sizeof(float4), &B->pair_full[b]);
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
    // ---------------- MMA issuer: D[buffer] = A(fixed) * B(streamed)^T ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_128x128();
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
          const uint32_t bBase = sS + s * kTileBytes;
#pragma unroll
          for (int kk = 0; kk < kK / 16; ++kk)
            umma_bf16(tmem + b * kTile, sdesc_sw128(sF + kk * 32), sdesc_sw128(bBase + kk * 32), idesc, kk > 0);
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
    // ---------------- epilogue: warps 0-7; lane index t, column half h ----------------
    const int t = (warp & 3) * 32 + lane;  // TMEM lane = row of D owned (0..127)
    const int h = warp >> 2;               // which 64 of the 128 accumulator columns
    const SweepParams sp = make_sweep_params(sweep_kappa(dev->kappa, k), k);
    const uint64_t ahA2 = pk(sp.ahA, sp.ahA), alA2 = pk(sp.alA, sp.alA);
    const float dal = (float)(sp.aB - sp.aA);  // stream B: v^B = (a^B - a^A) z + (v^A + dB)
    const uint64_t da2 = pk(dal, dal);
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;  // TMEM lane field
    // this thread's own offsets (G1: its row's shift; G2: its column's offset, negated,
    // and the column's dB as stored in the pair arrays)
    uint64_t ownA2, ownD2 = 0ull;
    const int64_t own = fixed0 + t;
    if (ROWS) {
      const float2 rq = w.rowshift[cur][own < n ? own : n - 1];
      ownA2 = pk(-rq.x, -rq.x);
    } else {
      const float4 cq = w.colq[cur][own];  // padded columns: {+inf, 0, +inf, 0}
      ownA2 = pk(-cq.x, -cq.x);
      // the column's dB = BqA - BcolB, the same float the row sweep reads (padding: -2^100)
      const float db = pair_dB(w.colq2[cur], own);
      ownD2 = pk(db, db);
    }
    float hiA = 0.f, loA = 0.f, hiB = 0.f, loB = 0.f, hiC = 0.f, loC = 0.f;
    // packed pair sums over this warp's 64 columns of a tile (two alternating accumulators)
    uint64_t accA[2], accB[2], accC[2];
    auto reset = [&]() {
      accA[0] = accA[1] = accB[0] = accB[1] = accC[0] = accC[1] = 0ull;
    };
    auto fold = [&]() {
      const float2 a2 = upk(f2add(accA[0], accA[1])), b2 = upk(f2add(accB[0], accB[1]));
      ff_add(hiA, loA, a2.x + a2.y);
      ff_add(hiB, loB, b2.x + b2.y);
      if (WC) {
        const float2 c2 = upk(f2add(accC[0], accC[1]));
        ff_add(hiC, loC, c2.x + c2.y);
      }
    };
    // 16 accumulator columns (8 pairs) starting at column col of the tile
    auto half_chunk = [&](const uint32_t (&v)[16], const float4* pr, int col) {
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        const float4 qa = pr[col + 2 * p];
        const float4 qb = pr[col + 2 * p + 1];
        const uint64_t z2 = pk(__uint_as_float(v[2 * p]), __uint_as_float(v[2 * p + 1]));
        const uint64_t vA = f2fma(alA2, z2, f2fma(ahA2, z2, f2add(ownA2, pk(qa.x, qa.y))));
        // G1: the inner column's BqA - BqB from the pair data; G2: the own column's
        const uint64_t vB = f2fma(da2, z2, f2add(vA, ROWS ? pk(qb.x, qb.y) : ownD2));
        const float2 vAf = upk(vA), vBf = upk(vB);
        const uint64_t eA = pk(ex2(vAf.x), ex2(vAf.y));
        const uint64_t eB = pk(ex2(vBf.x), ex2(vBf.y));
        if (WC) {
          const uint64_t pA = f2mul(eA, pk(qa.z, qa.w));
          accA[p & 1] = f2add(accA[p & 1], pA);
          accC[p & 1] = f2fma(z2, pA, accC[p & 1]);
        } else {
          accA[p & 1] = f2fma(eA, pk(qa.z, qa.w), accA[p & 1]);
        }
        // G1: stream B's column weight is inside dB; G2: weight by the row's q^B
        if (ROWS) accB[p & 1] = f2add(accB[p & 1], eB);
        else accB[p & 1] = f2fma(eB, pk(qb.z, qb.w), accB[p & 1]);
      }
    };
    for (int i = 0; i < ntiles; ++i) {
      const int b = i & 1;
      bool ok = mbar_wait(&B->pair_full[b], (i >> 1) & 1, B, dev);
      ok = ok && mbar_wait(&B->tmem_full[b], (i >> 1) & 1, B, dev);
      // warp-uniform decision before the .sync.aligned TMEM loads
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const float4* pr = sPair + (size_t)b * kTile;
      // this warp's 64 columns as two 32-column loads (each with its wait); other warps
      // of the SM sub-partition cover the TMEM latency
      const uint32_t tbase = tmem + lane_base + b * kTile + h * 64;
      reset();
#pragma unroll 1
      for (int c = 0; c < 2; ++c) {
        uint32_t v[32];
        tmem_ld32_wait(tbase + c * 32, v);
        half_chunk(*reinterpret_cast<const uint32_t(*)[16]>(&v[0]), pr, h * 64 + c * 32);
        half_chunk(*reinterpret_cast<const uint32_t(*)[16]>(&v[16]), pr, h * 64 + c * 32 + 16);
      }
      fold();
      tc_fence_before();
      mbar_arrive(&B->tmem_empty[b]);
      mbar_arrive(&B->pair_empty[b]);
    }
    // combine the two column halves of each lane (the stream ring is idle now: every
    // loaded tile has been consumed by an MMA whose completion the epilogue waited for)
    double* comb = reinterpret_cast<double*>(sStream);
    if (h == 1) {
      comb[t * 3 + 0] = (double)hiA + (double)loA;
      comb[t * 3 + 1] = (double)hiB + (double)loB;
      comb[t * 3 + 2] = (double)hiC + (double)loC;
    }
    epi_bar();
    if (h == 0 && !*(volatile int*)&B->err) {
      const double sA = (double)hiA + (double)loA + comb[t * 3 + 0];
      const double sB = (double)hiB + (double)loB + comb[t * 3 + 1];
      const double sC = (double)hiC + (double)loC + comb[t * 3 + 2];
      if (ROWS) {
        if (own < n) {
          w.rowpart[((int64_t)blockIdx.y * 2 + 0) * n + own] = sA;
          w.rowpart[((int64_t)blockIdx.y * 2 + 1) * n + own] = sB;
        }
      } else if (own < m) {
        constexpr int na = WC ? 3 : 2;  // the layout k_col_fin reads for this pass
        w.colpart[((int64_t)blockIdx.y * na + 0) * m + own] = sA;
        w.colpart[((int64_t)blockIdx.y * na + 1) * m + own] = sB;
        if (WC) w.colpart[((int64_t)blockIdx.y * na + 2) * m + own] = sC;
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
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
  // alignment slack + fixed tile + ring + barriers + packed pairs (2 x 128 float4)
  return 1024 + (size_t)tc::kTileBytes * (1 + tc::kStages) + tc::kBarBytes + 2 * tc::kTile * sizeof(float4);
}

int64_t tc_pad(int64_t v) { return (v + tc::kTile - 1) / tc::kTile * tc::kTile; }

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

// encode a 2-D bf16 tensor map over a (rows_pad x 64) row-major array, 128 x 64 boxes, 128B swizzle
cudaError_t tc_make_map(void* map_out, const void* base, int64_t rows_pad) {
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
  cuuint64_t dims[2] = {(cuuint64_t)tc::kK, (cuuint64_t)rows_pad};
  cuuint64_t strides[1] = {(cuuint64_t)tc::kK * 2};
  cuuint32_t box[2] = {(cuuint32_t)tc::kK, (cuuint32_t)tc::kTile};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_prepare() {
  const int sm = (int)tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(tc::k_tc_sweep<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc::k_tc_sweep<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc::k_tc_sweep<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

int tc_blocks_per_sm(int which) {
  int nb = 0;
  if (which == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tc::k_tc_sweep<true, 0>, tc::kThreads, tc_smem_bytes());
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tc::k_tc_sweep<false, 1>, tc::kThreads, tc_smem_bytes());
  // two 256-column TMEM allocations fill the 512 columns of an SM
  if (nb > 2) nb = 2;
  return nb > 0 ? nb : 1;
}

cudaError_t tc_launch_sweep(bool rows, int eval, const void* map_x, const void* map_y, const Work& w,
                            const Consts& k, int splits, cudaStream_t st) {
  const int64_t nfixed = rows ? k.n : k.m;
  const int64_t nstream = rows ? k.m : k.n;
  const int64_t ntiles = (nstream + tc::kTile - 1) / tc::kTile;
  const int tps = (int)((ntiles + splits - 1) / splits);
  dim3 grid((unsigned)((nfixed + tc::kTile - 1) / tc::kTile), (unsigned)splits);
  const CUtensorMap& mx = *reinterpret_cast<const CUtensorMap*>(map_x);
  const CUtensorMap& my = *reinterpret_cast<const CUtensorMap*>(map_y);
  if (rows)
    tc::k_tc_sweep<true, 0><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mx, my, w, k.n, k.m, tps, k);
  else if (eval)
    tc::k_tc_sweep<false, 1><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mx, my, w, k.n, k.m, tps, k);
  else
    tc::k_tc_sweep<false, 0><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mx, my, w, k.n, k.m, tps, k);
  return cudaGetLastError();
}

}  // namespace lamp
