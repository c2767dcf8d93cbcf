// Stored-cost sweeps fed by TMA: the row sweep G1 and the column sweep G2 of Alg. 2 over a
// dense float32 cost C (n x m, row-major, leading dimension ldc), one pass per sweep with
// both streams A (kappa_t, nu^t) and B (kappa_{t+1}, nubar^{t+1}) (Section 4.1).
//
// One producer warp streams 32-row x 256-column tiles of C (2-D tensor copies, 32 KB)
// together with the per-point data of the tile (G1: the 256 columns' {BqA, wA, BqB, wB};
// G2: the 32 rows' {RqA, qA, RqB, qB}, plain bulk copies) through a 3-stage shared-memory
// ring; eight consumer warps evaluate the compensated exponents of both streams and their
// ex2 in float32 and accumulate:
//   G1: warp w owns rows 4w .. 4w + 3 of the CTA's 32-row block, lane l the columns
//       l + 32 q (q < 8) of each tile; per-row float-float sums, one warp reduction at the
//       end, partials per column split;
//   G2: warp w owns the 32 columns 32 w .. 32 w + 31 of the CTA's 256-column block (one
//       per lane) and walks the 32 rows of each tile; partials per row split.
// The exponent of entry (i, j) is formed from the same operands in the same order in both
// sweeps, so G2 sums exactly the entries that G1 normalised.  Every wait is bounded
// (lamp_async.cuh).
#include <cuda.h>

#include <cmath>
#include <cstdint>

#include "lamp_async.cuh"
#include "lamp_common.cuh"

namespace lamp {

namespace dense {

constexpr int kTR = 32;                                  // rows of a tile
constexpr int kTC = 256;                                 // columns of a tile (TMA box inner extent)
constexpr int kStages = 3;
constexpr int kTileBytes = kTR * kTC * 4;                // 32 KiB
constexpr int kAuxMax = kTC;                             // float4 per-point data per stage (G1: 256)
constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kProducerWarp = kConsumerWarps;
constexpr int kThreads = kConsumers + 32;
static_assert(kConsumerWarps * 4 == kTR && kConsumerWarps * 32 == kTC, "warp / tile layout");

struct __align__(8) Bars {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  int err;
};

// tiles, per-point data, barriers, and slack to align the dynamic buffer to 128 bytes
constexpr size_t kSmemBytes = (size_t)kStages * kTileBytes + (size_t)kStages * kAuxMax * sizeof(float4) + 128 + 128;

template <bool ROWS, int WC>
__global__ void __launch_bounds__(kThreads, 2)
k_dense_tma(const __grid_constant__ CUtensorMap map_c, const Work w, int64_t n, int64_t m, int tiles_per_split,
            const Consts k) {
  DevState* __restrict__ dev = w.dev;
  if (dev->done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* sC = reinterpret_cast<float*>(smem);                                    // kStages x kTR x kTC
  float4* sAux = reinterpret_cast<float4*>(smem + (size_t)kStages * kTileBytes);  // kStages x kAuxMax
  Bars* B = reinterpret_cast<Bars*>(smem + (size_t)kStages * kTileBytes + (size_t)kStages * kAuxMax * 16);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int cur = dev->cur;
  const int64_t ntiles_all = ROWS ? (m + kTC - 1) / kTC : (n + kTR - 1) / kTR;
  const int64_t it0 = (int64_t)blockIdx.y * tiles_per_split;
  int64_t it1 = it0 + tiles_per_split;
  if (it1 > ntiles_all) it1 = ntiles_all;
  const int ntiles = it1 > it0 ? (int)(it1 - it0) : 0;
  constexpr int kAux = ROWS ? kTC : kTR;  // per-point data entries per tile

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      async::mbar_init(&B->full[s], 1);
      async::mbar_init(&B->empty[s], kConsumers);
    }
    B->err = 0;
    async::mbar_init_fence();
  }
  __syncthreads();

  if (warp == kProducerWarp) {
    if (lane == 0) {
      const float4* __restrict__ aux_src = ROWS ? w.colq[cur] : w.g2row;
      int issued = 0;
      for (int i = 0; i < ntiles; ++i) {
        const int s = i % kStages;
        if (i >= kStages && !async::mbar_wait(&B->empty[s], ((i / kStages) & 1) ^ 1, &B->err, dev)) break;
        const int64_t t = it0 + i;
        async::mbar_expect_tx(&B->full[s], kTileBytes + kAux * (uint32_t)sizeof(float4));
        if (ROWS) {
          async::tma_load_2d(sC + (size_t)s * kTR * kTC, &map_c, &B->full[s], (int)(t * kTC), (int)(blockIdx.x * kTR));
        } else {
          async::tma_load_2d(sC + (size_t)s * kTR * kTC, &map_c, &B->full[s], (int)(blockIdx.x * kTC), (int)(t * kTR));
        }
        // the per-point arrays are padded (columns to whole 256-column tiles, rows to
        // whole 128-row units) with entries whose offsets are +inf and weights 0, so the
        // entries past the end of C (read as 0 by the tensor copy) contribute 0
        async::bulk_load(sAux + (size_t)s * kAuxMax, aux_src + t * kAux, kAux * (uint32_t)sizeof(float4), &B->full[s]);
        issued = i + 1;
      }
      if (*(volatile int*)&B->err) {
        // error: let this thread's copies in flight land before the CTA exits
        for (int i = issued - kStages < 0 ? 0 : issued - kStages; i < issued; ++i)
          async::mbar_drain(&B->full[i % kStages], (i / kStages) & 1);
      }
    }
  } else {
    const SweepF sp = sweep_floats_of(dev, k);
    const float ahA = sp.ahA, alA = sp.alA, ahB = sp.ahB, alB = sp.alB;
    if (ROWS) {
      // ---------------- G1: rows 4 warp .. 4 warp + 3 of this row block ----------------
      float oA[4], oB[4];
      int64_t gi[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        gi[a] = (int64_t)blockIdx.x * kTR + 4 * warp + a;
        const float2 q = w.rowshift[cur][gi[a] < n ? gi[a] : n - 1];
        oA[a] = q.x;
        oB[a] = q.y;
      }
      float hA[4] = {0.f, 0.f, 0.f, 0.f}, lA[4] = {0.f, 0.f, 0.f, 0.f};
      float hB[4] = {0.f, 0.f, 0.f, 0.f}, lB[4] = {0.f, 0.f, 0.f, 0.f};
      bool ok = true;
      for (int i = 0; i < ntiles; ++i) {
        const int s = i % kStages;
        ok = async::mbar_wait(&B->full[s], (i / kStages) & 1, &B->err, dev);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        const float* tC = sC + (size_t)s * kTR * kTC + (size_t)(4 * warp) * kTC;
        const float4* tA = sAux + (size_t)s * kAuxMax;
        float sA[4] = {0.f, 0.f, 0.f, 0.f}, sB[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < kTC / 32; ++q) {
          const int col = lane + 32 * q;
          const float4 cd = tA[col];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float zz = tC[a * kTC + col];
            const float vA = __fmaf_rn(alA, zz, __fmaf_rn(ahA, zz, -(oA[a] + cd.x)));
            const float vB = __fmaf_rn(alB, zz, __fmaf_rn(ahB, zz, -(oB[a] + cd.z)));
            sA[a] = __fmaf_rn(ex2(vA), cd.y, sA[a]);
            sB[a] = __fmaf_rn(ex2(vB), cd.w, sB[a]);
          }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          ff_add(hA[a], lA[a], sA[a]);
          ff_add(hB[a], lB[a], sB[a]);
        }
        // the tile was read through the generic proxy; the next tensor copy into it is an
        // async-proxy write
        async::fence_proxy_async_smem();
        async::mbar_arrive(&B->empty[s]);
      }
      // warp-uniform: the reduction below needs every lane
      if (__all_sync(0xffffffffu, ok && !*(volatile int*)&B->err)) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          warp_sum_ff(hA[a], lA[a]);
          warp_sum_ff(hB[a], lB[a]);
          if (lane == 0 && gi[a] < n) {
            w.rowpart[((int64_t)blockIdx.y * 2 + 0) * n + gi[a]] = (double)hA[a] + (double)lA[a];
            w.rowpart[((int64_t)blockIdx.y * 2 + 1) * n + gi[a]] = (double)hB[a] + (double)lB[a];
          }
        }
      }
    } else {
      // ---------------- G2: column 32 warp + lane of this column block ----------------
      const int64_t gj = (int64_t)blockIdx.x * kTC + 32 * warp + lane;
      const int64_t mp = (m + 127) / 128 * 128;  // the column data are padded to mp
      const float4 cq = w.colq[cur][gj < mp ? gj : mp - 1];
      const float oA = cq.x, oB = cq.z;
      float hA = 0.f, lA = 0.f, hB = 0.f, lB = 0.f, hC = 0.f, lC = 0.f;
      bool ok = true;
      for (int i = 0; i < ntiles; ++i) {
        const int s = i % kStages;
        ok = async::mbar_wait(&B->full[s], (i / kStages) & 1, &B->err, dev);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        const float* tC = sC + (size_t)s * kTR * kTC + 32 * warp + lane;
        const float4* tR = sAux + (size_t)s * kAuxMax;
        float sA = 0.f, sB = 0.f, sCx = 0.f;
#pragma unroll 8
        for (int a = 0; a < kTR; ++a) {
          const float4 rd = tR[a];
          const float zz = tC[a * kTC];
          const float vA = __fmaf_rn(alA, zz, __fmaf_rn(ahA, zz, -(oA + rd.x)));
          const float vB = __fmaf_rn(alB, zz, __fmaf_rn(ahB, zz, -(oB + rd.z)));
          const float pA = ex2(vA) * rd.y;
          sA += pA;
          if (WC) sCx = __fmaf_rn(zz, pA, sCx);
          sB = __fmaf_rn(ex2(vB), rd.w, sB);
        }
        ff_add(hA, lA, sA);
        ff_add(hB, lB, sB);
        if (WC) ff_add(hC, lC, sCx);
        async::fence_proxy_async_smem();
        async::mbar_arrive(&B->empty[s]);
      }
      if (ok && !*(volatile int*)&B->err && gj < m) {
        constexpr int na = WC ? 3 : 2;  // the layout k_col_fin reads for this pass
        w.colpart[((int64_t)blockIdx.y * na + 0) * m + gj] = (double)hA + (double)lA;
        w.colpart[((int64_t)blockIdx.y * na + 1) * m + gj] = (double)hB + (double)lB;
        if (WC) w.colpart[((int64_t)blockIdx.y * na + 2) * m + gj] = (double)hC + (double)lC;
      }
    }
  }
  __syncthreads();
}

}  // namespace dense

// encode the float32 tensor map of a stored cost (n x m, leading dimension ldc floats):
// boxes of 32 rows x 256 columns; needs a 16-byte aligned base and ldc a multiple of 4
cudaError_t dense_make_map(void* map_out, const float* C, int64_t n, int64_t m, int64_t ldc) {
  if (reinterpret_cast<uintptr_t>(C) % 16 != 0 || ldc % 4 != 0 || ldc < m) return cudaErrorInvalidValue;
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
  cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ldc * 4};
  cuuint32_t box[2] = {(cuuint32_t)dense::kTC, (cuuint32_t)dense::kTR};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(C),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t dense_prepare() {
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)dense::k_dense_tma<true, 0>, (const void*)dense::k_dense_tma<false, 0>,
                        (const void*)dense::k_dense_tma<false, 1>}) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense::kSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  }
  return e;
}

int dense_tile_rows() { return dense::kTR; }
int dense_tile_cols() { return dense::kTC; }

int dense_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dense::k_dense_tma<false, 1>, dense::kThreads, dense::kSmemBytes);
  return nb > 0 ? nb : 1;
}

cudaError_t dense_launch_sweep(bool rows, int eval, const Geometry& g, const Work& w, const Consts& k, int splits,
                               cudaStream_t st) {
  const int64_t nblk = rows ? (k.n + dense::kTR - 1) / dense::kTR : (k.m + dense::kTC - 1) / dense::kTC;
  const int64_t ntiles = rows ? (k.m + dense::kTC - 1) / dense::kTC : (k.n + dense::kTR - 1) / dense::kTR;
  const int tps = (int)((ntiles + splits - 1) / splits);
  dim3 grid((unsigned)nblk, (unsigned)splits);
  const CUtensorMap& map = *reinterpret_cast<const CUtensorMap*>(g.map_c);
  if (rows)
    dense::k_dense_tma<true, 0><<<grid, dense::kThreads, dense::kSmemBytes, st>>>(map, w, k.n, k.m, tps, k);
  else if (eval)
    dense::k_dense_tma<false, 1><<<grid, dense::kThreads, dense::kSmemBytes, st>>>(map, w, k.n, k.m, tps, k);
  else
    dense::k_dense_tma<false, 0><<<grid, dense::kThreads, dense::kSmemBytes, st>>>(map, w, k.n, k.m, tps, k);
  return cudaGetLastError();
}

}  // namespace lamp
