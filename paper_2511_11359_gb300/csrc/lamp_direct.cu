// Packed f32x2 direct-form sweeps of the LAMP hot path (arXiv 2511.11359, Alg. 2,
// Section 4.1) for on-the-fly costs of low-dimensional point clouds (d <= 8): the row
// sweep G1 and the column sweep G2 of both streams, for the ground costs |x - y|^2,
// |x - y|_1 and |x - y|_inf (App. E.2 compares LAMP under all three).  See lamp_common.cuh for the
// compensated exponent and the shared row shift.
#include <cmath>
#include <cstdint>

#include "lamp_common.cuh"

namespace lamp {

namespace {

constexpr int kThreads = 256;
enum SweepMode : int { M_ROWSUM = 0, M_COLSUM = 1 };

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ------------------------------------------------------------------------------------------
// direct-form sweeps over point clouds with d <= 8 (LAMP_COST_SQEUCLID, float32, packed f32x2)
//
// Each thread owns kR(D) outer points o0 + tid + 256 r for the CTA's lifetime and
// keeps their coordinates and exponent offsets in registers as duplicated pairs
// (x, x).  The CTA streams the inner points through shared memory in tiles of 128
// (64 pairs, double-buffered with cp.async) and all threads read the same inner
// pair at the same time (broadcast loads), so one f32x2 instruction serves the two
// entries (outer, 2p) and (outer, 2p + 1).  Per pair of entries: d subtractions
// and d multiply-adds for z = |x - y|^2; stream A one add, two fma (compensated
// exponent), two ex2 and one fma (weighted sum); stream B, through the shared row
// shift (see lamp_common.cuh), one add, one fma, two ex2 and one add (row sums) or
// fma (column sums).  Evaluation
// passes also accumulate sum_i z_ij X_ij in the column sweep (two more).
// z = sum_k (x_k - y_k)^2 is accumulated in the same k order in both sweeps, and
// (y - x)^2 == (x - y)^2 in IEEE arithmetic, so the row and the column sweep see
// bit-identical exponents.  The inner data are the packed-pair arrays (see Work).

constexpr int kDTile = kDirectTile;  // inner points per shared-memory tile
constexpr int kDPairs = kDTile / 2;  // pairs per tile
constexpr int kDFold = 32;           // pairs between float-float folds of the packed sums

template <int D>
struct DirectCfg {
  static constexpr int R = D <= 4 ? 4 : 2;  // outer points per thread
  static constexpr int DP = (D + 1) & ~1;   // coordinates per pair record, even
  static constexpr int REC = DP * 2 + 8;    // floats per pair record: coords [DP][2], offsets/weights A, B
  static constexpr int OUTER = kThreads * R;
};

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// stage inner tile `it` (points it*128 ..) into the record buffer `rec`
template <int D>
__device__ __forceinline__ void direct_stage(float* rec, const float* __restrict__ P_in, int64_t n_in,
                                             const float4* __restrict__ pairs, int64_t it, int tid) {
  using C = DirectCfg<D>;
  const int64_t i0 = it * kDTile;
  for (int idx = tid; idx < kDTile * D; idx += kThreads) {
    const int b = idx / D, k = idx - (idx / D) * D;
    const bool ok = i0 + b < n_in;
    const float* src = ok ? P_in + (i0 + b) * D + k : P_in;
    cp_async4(rec + (b >> 1) * C::REC + k * 2 + (b & 1), src, ok);
  }
  // offsets / weights: pairs [2(i0/2 + p)] (stream A) and [2(i0/2 + p) + 1] (stream B);
  // the pair arrays are padded to 128 entries, so a whole tile is always in bounds
  for (int idx = tid; idx < kDPairs * 2; idx += kThreads) {
    const int p = idx >> 1, s = idx & 1;
    cp_async16(rec + p * C::REC + C::DP * 2 + 4 * s, pairs + (i0 >> 1) * 2 + idx);
  }
}

// |x_k - y_k| for a pair of entries: clear both sign bits
__device__ __forceinline__ uint64_t f2abs(uint64_t v) {
  uint64_t r;
  asm("and.b64 %0, %1, 0x7FFFFFFF7FFFFFFF;" : "=l"(r) : "l"(v));
  return r;
}
__device__ __forceinline__ uint64_t f2max(uint64_t a, uint64_t b) {
  const float2 x = upk(a), y = upk(b);
  return pk(fmaxf(x.x, y.x), fmaxf(x.y, y.y));
}

// MODE = M_ROWSUM, or M_COLSUM with WC = 1 (evaluation pass: cost-weighted column sums too) or 0;
// CK = the ground cost (Consts::cost_op): 0 |x - y|^2, 1 l1, 2 l-inf
template <int MODE, int D, int WC, int CK>
__global__ void __launch_bounds__(kThreads, 2)
k_pts_direct(const float* __restrict__ P_out, const float* __restrict__ P_in, int64_t n_out, int64_t n_in,
             const Work w, double* __restrict__ part, int tiles_per_split, const Consts k) {
  using C = DirectCfg<D>;
  constexpr int R = C::R, DP = C::DP, REC = C::REC;
  constexpr int NACC = WC ? 3 : 2;
  const DevState* __restrict__ dev = w.dev;
  if (dev->done) return;
  const int cur = dev->cur;
  // row sweep: inner = columns (colq2 of the current state); column sweep: inner = rows (g2row2)
  const float4* __restrict__ pairs = MODE == M_ROWSUM ? w.colq2[cur] : w.g2row2;
  __shared__ __align__(16) float srec[2][kDPairs * REC];

  const int tid = threadIdx.x;
  const int64_t o0 = (int64_t)blockIdx.x * C::OUTER;
  const int split = blockIdx.y;
  const int64_t ntiles = (n_in + kDTile - 1) / kDTile;
  const int64_t it0 = (int64_t)split * tiles_per_split;
  const int64_t it1 = it0 + tiles_per_split < ntiles ? it0 + tiles_per_split : ntiles;

  if (it0 < it1) direct_stage<D>(srec[0], P_in, n_in, pairs, it0, tid);
  cp_async_commit();
  if (DP > D) {  // the padding coordinate of odd d is read by the 16-byte loads, never used
    for (int p = tid; p < 2 * kDPairs; p += kThreads) {
      srec[p / kDPairs][(p % kDPairs) * REC + 2 * D] = 0.f;
      srec[p / kDPairs][(p % kDPairs) * REC + 2 * D + 1] = 0.f;
    }
  }

  const SweepF sp = sweep_floats_of(dev, k);
  const uint64_t ahA2 = pk(sp.ahA, sp.ahA), alA2 = pk(sp.alA, sp.alA);
  const float dal = sp.dal;  // a^B - a^A
  const uint64_t da2 = pk(dal, dal);

  // own offsets: -RqA_i (row sweep), or -BqA_j and dB_j = BqA_j - BqB_j (column sweep)
  uint64_t x2[R][D], ownA[R], ownD[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int64_t go = o0 + tid + (int64_t)kThreads * r;
    if (go >= n_out) go = n_out - 1;
#pragma unroll
    for (int kk = 0; kk < D; ++kk) {
      const float v = P_out[go * D + kk];
      x2[r][kk] = pk(v, v);
    }
    float qa, db = 0.f;
    if (MODE == M_ROWSUM) {
      qa = w.rowshift[cur][go].x;
    } else {
      qa = w.colq[cur][go].x;
      db = pair_dB(w.colq2[cur], go);  // the same float the row sweep reads for this column
    }
    ownA[r] = pk(-qa, -qa);
    ownD[r] = pk(db, db);
  }

  float hi[R][NACC], lo[R][NACC];
  uint64_t acc[R][NACC];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < NACC; ++q) {
      hi[r][q] = 0.f;
      lo[r][q] = 0.f;
      acc[r][q] = 0ull;  // (+0, +0)
    }

  for (int64_t it = it0; it < it1; ++it) {
    const int buf = (int)((it - it0) & 1);
    if (it + 1 < it1) direct_stage<D>(srec[buf ^ 1], P_in, n_in, pairs, it + 1, tid);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const float* rec = srec[buf];
#pragma unroll 1
    for (int p0 = 0; p0 < kDPairs; p0 += kDFold) {
#pragma unroll 2
      for (int p = p0; p < p0 + kDFold; ++p) {
        const float* rp = rec + p * REC;
        uint64_t y2[DP];
#pragma unroll
        for (int kk = 0; kk < DP; kk += 2) {
          const float4 t = *reinterpret_cast<const float4*>(rp + 2 * kk);
          y2[kk] = pk(t.x, t.y);
          y2[kk + 1] = pk(t.z, t.w);
        }
        const float4 dA = *reinterpret_cast<const float4*>(rp + 2 * DP);
        const float4 dB = *reinterpret_cast<const float4*>(rp + 2 * DP + 4);
        const uint64_t oA2 = pk(dA.x, dA.y), wA2 = pk(dA.z, dA.w);
        const uint64_t wB2 = pk(dB.z, dB.w);
        // row sweep: the inner columns' dB_j = BqA_j - BcolB_j from the pair data
        const uint64_t dC2 = pk(dB.x, dB.y);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          uint64_t z2;
          if constexpr (CK == 0) {
            uint64_t df = f2sub(x2[r][0], y2[0]);
            z2 = f2mul(df, df);
#pragma unroll
            for (int kk = 1; kk < D; ++kk) {
              df = f2sub(x2[r][kk], y2[kk]);
              z2 = f2fma(df, df, z2);
            }
          } else {
            z2 = f2abs(f2sub(x2[r][0], y2[0]));
#pragma unroll
            for (int kk = 1; kk < D; ++kk) {
              const uint64_t ad = f2abs(f2sub(x2[r][kk], y2[kk]));
              z2 = CK == 1 ? f2add(z2, ad) : f2max(z2, ad);
            }
          }
          const uint64_t vA = f2fma(alA2, z2, f2fma(ahA2, z2, f2add(ownA[r], oA2)));
          const uint64_t vB = f2fma(da2, z2, f2add(vA, MODE == M_ROWSUM ? dC2 : ownD[r]));
          const float2 vAf = upk(vA), vBf = upk(vB);
          const uint64_t eA = pk(ex2(vAf.x), ex2(vAf.y));
          const uint64_t eB = pk(ex2(vBf.x), ex2(vBf.y));
          if constexpr (WC) {
            const uint64_t pA = f2mul(eA, wA2);
            acc[r][0] = f2add(acc[r][0], pA);
            acc[r][2] = f2fma(z2, pA, acc[r][2]);
          } else {
            acc[r][0] = f2fma(eA, wA2, acc[r][0]);
          }
          // row sums of stream B carry no weight (it is inside dB_j); column sums weight by q^B_i
          if constexpr (MODE == M_ROWSUM) acc[r][1] = f2add(acc[r][1], eB);
          else acc[r][1] = f2fma(eB, wB2, acc[r][1]);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < NACC; ++q) {
          const float2 s = upk(acc[r][q]);
          ff_add(hi[r][q], lo[r][q], s.x + s.y);
          acc[r][q] = 0ull;
        }
    }
    __syncthreads();  // every thread is done with srec[buf] before it is refilled
  }
  cp_async_wait<0>();

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t go = o0 + tid + (int64_t)kThreads * r;
    if (go >= n_out) continue;
#pragma unroll
    for (int q = 0; q < NACC; ++q) part[((int64_t)split * NACC + q) * n_out + go] = (double)hi[r][q] + (double)lo[r][q];
  }
}

template <int MODE, int D, int WC, int CK>
static cudaError_t launch_direct_d(const float* Pout, const float* Pin, int64_t nout, int64_t nin, const Work& w,
                                   double* part, int splits, const Consts& k, cudaStream_t st) {
  int64_t tin = cdiv(nin, kDTile);
  int tps = (int)cdiv(tin, splits);
  dim3 grid((unsigned)cdiv(nout, DirectCfg<D>::OUTER), (unsigned)splits);
  k_pts_direct<MODE, D, WC, CK><<<grid, kThreads, 0, st>>>(Pout, Pin, nout, nin, w, part, tps, k);
  return cudaGetLastError();
}

template <int MODE, int WC, int CK>
static cudaError_t launch_direct_ck(const float* Pout, const float* Pin, int64_t nout, int64_t nin, const Work& w,
                                    double* part, int splits, const Consts& k, cudaStream_t st) {
  switch (k.d) {
    case 1: return launch_direct_d<MODE, 1, WC, CK>(Pout, Pin, nout, nin, w, part, splits, k, st);
    case 2: return launch_direct_d<MODE, 2, WC, CK>(Pout, Pin, nout, nin, w, part, splits, k, st);
    case 3: return launch_direct_d<MODE, 3, WC, CK>(Pout, Pin, nout, nin, w, part, splits, k, st);
    case 4: return launch_direct_d<MODE, 4, WC, CK>(Pout, Pin, nout, nin, w, part, splits, k, st);
    case 5: return launch_direct_d<MODE, 5, WC, CK>(Pout, Pin, nout, nin, w, part, splits, k, st);
    case 6: return launch_direct_d<MODE, 6, WC, CK>(Pout, Pin, nout, nin, w, part, splits, k, st);
    case 7: return launch_direct_d<MODE, 7, WC, CK>(Pout, Pin, nout, nin, w, part, splits, k, st);
    case 8: return launch_direct_d<MODE, 8, WC, CK>(Pout, Pin, nout, nin, w, part, splits, k, st);
    default: return cudaErrorNotSupported;
  }
}

template <int MODE, int WC>
static cudaError_t launch_direct(const float* Pout, const float* Pin, int64_t nout, int64_t nin, const Work& w,
                                 double* part, int splits, const Consts& k, cudaStream_t st) {
  switch (k.cost_op) {
    case 0: return launch_direct_ck<MODE, WC, 0>(Pout, Pin, nout, nin, w, part, splits, k, st);
    case 1: return launch_direct_ck<MODE, WC, 1>(Pout, Pin, nout, nin, w, part, splits, k, st);
    case 2: return launch_direct_ck<MODE, WC, 2>(Pout, Pin, nout, nin, w, part, splits, k, st);
    default: return cudaErrorNotSupported;
  }
}


}  // namespace

int direct_outer(int d) { return kThreads * (d <= 4 ? DirectCfg<4>::R : DirectCfg<8>::R); }

int direct_blocks_per_sm() {
  // every instantiation is declared with __launch_bounds__(kThreads, 2) and static shared memory
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pts_direct<M_COLSUM, 8, 1, 0>, kThreads, 0);
  return nb > 0 ? nb : 1;
}

cudaError_t launch_direct_sweep(bool rows, int eval, const Inputs& in, const Consts& k, const Work& w,
                                const Geometry& g, cudaStream_t st) {
  if (rows) return launch_direct<M_ROWSUM, 0>(in.x, in.y, k.n, k.m, w, w.rowpart, g.rows_split, k, st);
  if (eval) return launch_direct<M_COLSUM, 1>(in.y, in.x, k.m, k.n, w, w.colpart, g.cols_split, k, st);
  return launch_direct<M_COLSUM, 0>(in.y, in.x, k.m, k.n, w, w.colpart, g.cols_split, k, st);
}

}  // namespace lamp
