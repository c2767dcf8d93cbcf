// tcgen05 (5th-generation tensor core) sweeps of the LAMP hot path for the
// squared-Euclidean cost in dot form, BF16 points, FP32 accumulation in TMEM.
//
// Both sweeps of an iteration (row sums G1, column sums G2; Section 4.1) issue
// the SAME MMA for every (row tile, column tile) pair,
//     D[128 rows x 128 cols] = Xb[rows, 0:64] * Yb[cols, 0:64]^T
// (A = 128 points of x, B = 128 points of y, both K-major bf16 tiles staged by
// TMA with 128-byte swizzle), so that the z = x.y values the two sweeps see are
// bit-identical and the column sweep's normalisation matches the row sweep's
// sums exactly.  G1 keeps its x tile fixed and streams y tiles; G2 keeps its y
// tile fixed and streams x tiles.
//
// CTA = 6 warps: warps 0-3 read TMEM (warp w owns lanes 32w..32w+31, one row of
// D per thread) and do the exponent / ex2 / reduction epilogue, warp 4 issues
// TMA loads, warp 5 issues tcgen05.mma.  Two TMEM accumulators (2 x 128 columns)
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
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 256;         // two 128-column FP32 accumulators
constexpr uint32_t kWaitLimit = 1u << 24;   // bounded spin on every mbarrier
constexpr int kTimeoutStatus = 6;           // LAMP_E_TIMEOUT

struct __align__(8) Bars {
  uint64_t fixed_full;
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t tmem_full[2];
  uint64_t tmem_empty[2];
  uint32_t tmem_base;
  int err;
};

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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, Bars* B, DevState* dev) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
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

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes, one lane per thread
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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

// exchange-and-add butterfly: on entry every lane holds v[0..31] for 32 columns
// (its own row); on exit lane l holds in v[0] the sum over the 32 lanes of column l.
__device__ __forceinline__ float lane_column_sum(float (&v)[32], int lane) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = upper ? v[i] : v[i + off];
      const float keep = upper ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// ROWS = true: G1 (fixed x tile, streamed y tiles, per-row sums of both streams)
// ROWS = false: G2 (fixed y tile, streamed x tiles, per-column sums of both streams and
// of z * X for <C, X>)
template <bool ROWS>
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
  float* sColOff = reinterpret_cast<float*>(B + 1);         // G2: {BqA, BqB} x 128
  double* sRed = reinterpret_cast<double*>(sColOff + 2 * kTile);  // G2: [4 warps][3][128]

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
      mbar_init(&B->tmem_empty[b], 128);
    }
    B->err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (!ROWS) {
    // fixed column offsets of this CTA's 128 columns (BqA, BqB); padded columns hold +inf
    const float4* __restrict__ colq = w.colq[cur];
    for (int t = threadIdx.x; t < kTile; t += blockDim.x) {
      const float4 q = colq[fixed0 + t];
      sColOff[2 * t] = q.x;
      sColOff[2 * t + 1] = q.z;
    }
  }
  if (warp == 0) {
    tmem_alloc(&B->tmem_base, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = B->tmem_base;

  if (warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      mbar_expect_tx(&B->fixed_full, kTileBytes);
      tma_load_2d(sFixed, ROWS ? &map_x : &map_y, &B->fixed_full, 0, (int)fixed0);
      for (int i = 0; i < ntiles; ++i) {
        const int s = i % kStages;
        if (i >= kStages && !mbar_wait(&B->empty[s], ((i / kStages) & 1) ^ 1, B, dev)) break;
        mbar_expect_tx(&B->full[s], kTileBytes);
        tma_load_2d(sStream + s * kTileBytes, ROWS ? &map_y : &map_x, &B->full[s], 0, (int)((it0 + i) * kTile));
        issued = i + 1;
      }
      if (*(volatile int*)&B->err) {
        // error: let this thread's copies in flight land before the CTA exits
        mbar_drain(&B->fixed_full, 0);
        for (int i = issued - kStages < 0 ? 0 : issued - kStages; i < issued; ++i)
          mbar_drain(&B->full[i % kStages], (i / kStages) & 1);
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
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
          const uint32_t aBase = ROWS ? sF : sS + s * kTileBytes;
          const uint32_t bBase = ROWS ? sS + s * kTileBytes : sF;
#pragma unroll
          for (int kk = 0; kk < kK / 16; ++kk)
            umma_bf16(tmem + b * kTile, sdesc_sw128(aBase + kk * 32), sdesc_sw128(bBase + kk * 32), idesc, kk > 0);
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
    // ---------------- epilogue: warps 0-3, thread = row of D ----------------
    const SweepParams sp = make_sweep_params(dev->kappa, k);
    const float ahA = sp.ahA, alA = sp.alA, ahB = sp.ahB, alB = sp.alB;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    if (ROWS) {
      int64_t row = fixed0 + warp * 32 + lane;
      const int64_t rowc = row < n ? row : n - 1;
      const float2 rq = w.rowshift[cur][rowc];
      const float4* __restrict__ colq = w.colq[cur];
      float hiA = 0.f, loA = 0.f, hiB = 0.f, loB = 0.f;
      for (int i = 0; i < ntiles; ++i) {
        const int b = i & 1;
        // warp-uniform decision before the .sync.aligned TMEM loads
        if (!__all_sync(0xffffffffu, mbar_wait(&B->tmem_full[b], (i >> 1) & 1, B, dev))) break;
        tc_fence_after();
        const int64_t col0 = (it0 + i) * kTile;
#pragma unroll 1
        for (int c = 0; c < kTile / 32; ++c) {
          uint32_t v[32];
          tmem_ld32(tmem + lane_base + b * kTile + c * 32, v);
          tmem_wait_ld();
          float sA = 0.f, sB = 0.f;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float z = __uint_as_float(v[j]);
            const float4 cq = __ldg(colq + col0 + c * 32 + j);  // padded columns: {+inf, 0, +inf, 0}
            const float vA = __fmaf_rn(alA, z, __fmaf_rn(ahA, z, -(rq.x + cq.x)));
            const float vB = __fmaf_rn(alB, z, __fmaf_rn(ahB, z, -(rq.y + cq.z)));
            sA = __fmaf_rn(ex2(vA), cq.y, sA);
            sB = __fmaf_rn(ex2(vB), cq.w, sB);
          }
          ff_add(hiA, loA, sA);
          ff_add(hiB, loB, sB);
        }
        tc_fence_before();
        mbar_arrive(&B->tmem_empty[b]);
      }
      if (row < n && !*(volatile int*)&B->err) {
        w.rowpart[((int64_t)blockIdx.y * 2 + 0) * n + row] = (double)hiA + (double)loA;
        w.rowpart[((int64_t)blockIdx.y * 2 + 1) * n + row] = (double)hiB + (double)loB;
      }
    } else {
      // per-lane accumulators of the columns this lane ends up owning after the butterfly
      float hA[kTile / 32], lA[kTile / 32], hB[kTile / 32], lB[kTile / 32], hC[kTile / 32], lC[kTile / 32];
#pragma unroll
      for (int c = 0; c < kTile / 32; ++c) hA[c] = lA[c] = hB[c] = lB[c] = hC[c] = lC[c] = 0.f;
      for (int i = 0; i < ntiles; ++i) {
        const int b = i & 1;
        const int64_t row = (it0 + i) * kTile + warp * 32 + lane;
        const float4 rd = w.g2row[row];  // padded rows: {+inf, 0, +inf, 0}
        if (!__all_sync(0xffffffffu, mbar_wait(&B->tmem_full[b], (i >> 1) & 1, B, dev))) break;
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < kTile / 32; ++c) {
          uint32_t v[32];
          tmem_ld32(tmem + lane_base + b * kTile + c * 32, v);
          tmem_wait_ld();
          float p[32], pc[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float z = __uint_as_float(v[j]);
            const float coA = sColOff[2 * (c * 32 + j)];
            const float vA = __fmaf_rn(alA, z, __fmaf_rn(ahA, z, -(rd.x + coA)));
            p[j] = ex2(vA) * rd.y;
            pc[j] = z * p[j];
          }
          ff_add(hA[c], lA[c], lane_column_sum(p, lane));
          ff_add(hC[c], lC[c], lane_column_sum(pc, lane));
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float z = __uint_as_float(v[j]);
            const float coB = sColOff[2 * (c * 32 + j) + 1];
            const float vB = __fmaf_rn(alB, z, __fmaf_rn(ahB, z, -(rd.z + coB)));
            p[j] = ex2(vB) * rd.w;
          }
          ff_add(hB[c], lB[c], lane_column_sum(p, lane));
        }
        tc_fence_before();
        mbar_arrive(&B->tmem_empty[b]);
      }
      // cross-warp reduction of the 4 warps' column partials
#pragma unroll
      for (int c = 0; c < kTile / 32; ++c) {
        const int col = c * 32 + lane;
        sRed[(warp * 3 + 0) * kTile + col] = (double)hA[c] + (double)lA[c];
        sRed[(warp * 3 + 1) * kTile + col] = (double)hB[c] + (double)lB[c];
        sRed[(warp * 3 + 2) * kTile + col] = (double)hC[c] + (double)lC[c];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (!ROWS && threadIdx.x < kTile && !*(volatile int*)&B->err) {
    const int col = threadIdx.x;
    const int64_t gcol = fixed0 + col;
    if (gcol < m) {
      for (int q = 0; q < 3; ++q) {
        double s = 0.0;
        for (int wi = 0; wi < 4; ++wi) s += sRed[(wi * 3 + q) * kTile + col];
        w.colpart[((int64_t)blockIdx.y * 3 + q) * m + gcol] = s;
      }
    }
  }
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

}  // namespace tc

size_t tc_smem_bytes() {
  return 1024 /* alignment slack */ + (size_t)tc::kTileBytes * (1 + tc::kStages) + sizeof(tc::Bars) +
         2 * tc::kTile * sizeof(float) + 4 * 3 * tc::kTile * sizeof(double);
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
  cudaError_t e = cudaFuncSetAttribute(tc::k_tc_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc::k_tc_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes());
}

int tc_blocks_per_sm(int which) {
  int nb = 0;
  if (which == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tc::k_tc_sweep<true>, tc::kThreads, tc_smem_bytes());
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tc::k_tc_sweep<false>, tc::kThreads, tc_smem_bytes());
  // two 256-column TMEM allocations fill the 512 columns of an SM
  if (nb > 2) nb = 2;
  return nb > 0 ? nb : 1;
}

cudaError_t tc_launch_sweep(bool rows, const void* map_x, const void* map_y, const Work& w, const Consts& k,
                            int splits, cudaStream_t st) {
  const int64_t nfixed = rows ? k.n : k.m;
  const int64_t nstream = rows ? k.m : k.n;
  const int64_t ntiles = (nstream + tc::kTile - 1) / tc::kTile;
  const int tps = (int)((ntiles + splits - 1) / splits);
  dim3 grid((unsigned)((nfixed + tc::kTile - 1) / tc::kTile), (unsigned)splits);
  const CUtensorMap& mx = *reinterpret_cast<const CUtensorMap*>(map_x);
  const CUtensorMap& my = *reinterpret_cast<const CUtensorMap*>(map_y);
  if (rows)
    tc::k_tc_sweep<true><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mx, my, w, k.n, k.m, tps, k);
  else
    tc::k_tc_sweep<false><<<grid, tc::kThreads, tc_smem_bytes(), st>>>(mx, my, w, k.n, k.m, tps, k);
  return cudaGetLastError();
}

}  // namespace lamp
