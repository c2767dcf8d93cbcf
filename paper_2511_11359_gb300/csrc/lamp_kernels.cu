// CUDA kernels of the LAMP hot path (arXiv 2511.11359, Alg. 2 and Section 4).
//
// One iteration = four launches:
//   G1  row sweep     S^A_i, S^B_i = sum_j 2^{v_ij} w_j          (row LSE, Section 4.1)
//   RF  row finalize  log Z_i, weights q_i = r_i / S_i, next row shifts
//   G2  column sweep  col_j = w_j sum_i 2^{v_ij} q_i for both streams, and
//                     sum_i z_ij X_ij for <C, X^t>                 (column sum, Section 4.1)
//   CF  column finalize: the O(m) float64 dual step of Alg. 2 (thetabar, nu, thetahat,
//                     tclip), residual ||col - c||_1, the next sweep's column data; its
//                     last block reduces the block partials and applies or rejects the update.
// See lamp_common.cuh for the compensated exponent.
#include <cfloat>
#include <cmath>

#include "lamp_common.cuh"

namespace lamp {

// ------------------------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------------------------------------------------
// sweeps over point clouds (LAMP_COST_SQEUCLID, float32 CUDA-core x.y)

// stage a tile of 128 points (rows base.., np valid) x d coordinates into s[kk * 128 + p]:
// thread (p = idx % 128, coordinate quad) reads up to 4 consecutive coordinates of one
// point (one 16-byte load when d % 4 == 0) and consecutive threads write consecutive p,
// so the transposed shared stores are free of bank conflicts
__device__ __forceinline__ void stage_points(float* __restrict__ s, const float* __restrict__ P, int64_t base,
                                             int64_t np, int d, int tid, int nthreads) {
  const int dq = (d + 3) >> 2;
  for (int idx = tid; idx < 128 * dq; idx += nthreads) {
    const int p = idx & 127, kq = (idx >> 7) << 2;
    const int64_t g = base + p;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (g < np) {
      if ((d & 3) == 0) {
        const float4 t = *reinterpret_cast<const float4*>(P + g * d + kq);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (kq + q < d) v[q] = P[g * d + kq + q];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (kq + q < d) s[(kq + q) * 128 + p] = v[q];
  }
}
//
// A CTA of 256 threads owns 128 "outer" points and loops over tiles of 128
// "inner" points; each thread computes an 8x8 block of z = x.y (outer rows
// {4ty..4ty+3, 64+4ty..}, inner columns {4tx..4tx+3, 64+4tx..}), in a fixed
// k order so that the row sweep and the column sweep produce bit-identical z.
// Row sweep: outer = rows (x), inner = columns (y).  Column sweep: the reverse.

constexpr int kPT = 128;
constexpr int kThreads = 256;

// M_MAX2: row maxima of u_ij = v_ij - Br_j with the row shifts applied and the column
// remainders Br_j (floats, in the column data's second field) subtracted: the refinement
// pass of the eta = 0 dual bound (see launch_dual), accurate to a few ulps of the grid
enum SweepMode : int { M_ROWSUM = 0, M_COLSUM = 1, M_MAX = 2, M_KMAX = 3, M_GRAD = 4, M_MAX2 = 5 };

// buffers of a sweep, indexed by the state-buffer parity dev->cur
struct SweepIO {
  const float2* off2[2];
  const float4* off4[2];
  const float4* indat[2];
};

// M_GRAD accumulates sum_b 2^{v_ab} weight_b V_b[0:DG] with V = Vin (n_in x DG, row-major)
// when given, else coordinates q0 .. q0 + DG - 1 of the inner points (the gradient)
template <int MODE, int DG, bool DIFF>
__global__ void __launch_bounds__(kThreads, MODE == M_GRAD ? 1 : 2)
k_pts_sweep(const float* __restrict__ P_out, const float* __restrict__ P_in, int64_t n_out, int64_t n_in, int d,
            const SweepIO io, double* __restrict__ part, float* __restrict__ pmax, int tiles_per_split,
            const DevState* __restrict__ dev, const Consts k, const float* __restrict__ Vin, int q0) {
  if ((MODE == M_ROWSUM || MODE == M_COLSUM) && dev->done) return;
  const int cur = dev->cur;
  const float2* __restrict__ off2 = cur ? io.off2[1] : io.off2[0];
  const float4* __restrict__ off4 = cur ? io.off4[1] : io.off4[0];
  const float4* __restrict__ in_data = cur ? io.indat[1] : io.indat[0];
  extern __shared__ __align__(16) float smem[];
  float* sOut = smem;                          // [d][128]
  float* sIn = smem + d * kPT;                 // [d][128]
  float4* sDat = reinterpret_cast<float4*>(smem + 2 * d * kPT);  // [128]
  float* sV = smem + 2 * d * kPT + 4 * kPT;                        // [DG][128] (M_GRAD with Vin)

  const int tid = threadIdx.x;
  const int tx = tid & 15;
  const int ty = tid >> 4;
  const int64_t o0 = (int64_t)blockIdx.x * kPT;
  const int split = blockIdx.y;
  const int64_t ntiles_in = (n_in + kPT - 1) / kPT;
  const int64_t it0 = (int64_t)split * tiles_per_split;
  int64_t it1 = it0 + tiles_per_split;
  if (it1 > ntiles_in) it1 = ntiles_in;

  const SweepF sp = sweep_floats_of(dev, k);

  stage_points(sOut, P_out, o0, n_out, d, tid, kThreads);

  // outer offsets of this thread's 8 outer points
  float oA[8], oB[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    int64_t go = o0 + ((a < 4) ? (ty * 4 + a) : (64 + ty * 4 + a - 4));
    if (go >= n_out) go = n_out - 1;
    if (MODE == M_COLSUM) {
      float4 q = off4[go];
      oA[a] = q.x;
      oB[a] = q.z;
    } else if (MODE == M_GRAD) {
      float4 q = off4[go];  // row gradient: g2row {RqA, ..}; column gradient: colq {BqA, ..}
      oA[a] = q.x;
      oB[a] = 0.f;
    } else if (MODE == M_MAX) {
      oA[a] = 0.f;
      oB[a] = 0.f;
    } else if (MODE == M_MAX2) {
      oA[a] = off2[go].x;
      oB[a] = 0.f;
    } else {
      float2 q = off2[go];
      oA[a] = q.x;
      oB[a] = q.y;
    }
  }

  const float ahA = sp.ahA, alA = sp.alA, ahB = sp.ahB, alB = sp.alB;

  constexpr int NACC = (MODE == M_COLSUM) ? 3 : 2;
  float hi[8][NACC], lo[8][NACC];
  float mx[8][2];
  double gacc[8][DG > 0 ? DG : 1];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
#pragma unroll
    for (int q = 0; q < NACC; ++q) { hi[a][q] = 0.f; lo[a][q] = 0.f; }
    mx[a][0] = -INFINITY;
    mx[a][1] = -INFINITY;
#pragma unroll
    for (int q = 0; q < (DG > 0 ? DG : 1); ++q) gacc[a][q] = 0.0;
  }

  for (int64_t it = it0; it < it1; ++it) {
    const int64_t i0 = it * kPT;
    __syncthreads();
    stage_points(sIn, P_in, i0, n_in, d, tid, kThreads);
    if (MODE == M_GRAD && Vin) {
      for (int idx = tid; idx < DG * kPT; idx += kThreads) {
        int p = idx / (DG > 0 ? DG : 1), q = idx - p * (DG > 0 ? DG : 1);
        int64_t gi = i0 + p;
        sV[q * kPT + p] = gi < n_in ? Vin[gi * DG + q] : 0.0f;
      }
    }
    if (tid < kPT) {
      int64_t gi = i0 + tid;
      float4 v;
      if (gi < n_in) {
        v = in_data[gi];
      } else {
        v = make_float4(INFINITY, 0.f, INFINITY, 0.f);
        if (MODE == M_KMAX) v.x = -INFINITY;
      }
      sDat[tid] = v;
    }
    __syncthreads();

    float z[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) z[a][b] = 0.f;

#pragma unroll 2
    for (int kk = 0; kk < d; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&sOut[kk * kPT + ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&sOut[kk * kPT + 64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&sIn[kk * kPT + tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&sIn[kk * kPT + 64 + tx * 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
      if (DIFF) {
        // the ground cost of the direct form (Consts::cost_op; uniform branch)
        if (k.cost_op == 0) {
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) {
              const float df = av[a] - bv[b];
              z[a][b] = __fmaf_rn(df, df, z[a][b]);
            }
        } else if (k.cost_op == 1) {
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) z[a][b] += fabsf(av[a] - bv[b]);
        } else {
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) z[a][b] = fmaxf(z[a][b], fabsf(av[a] - bv[b]));
        }
      } else {
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) z[a][b] = __fmaf_rn(av[a], bv[b], z[a][b]);
      }
    }

    float4 dat[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) dat[b] = sDat[(b < 4) ? (tx * 4 + b) : (64 + tx * 4 + b - 4)];

    if (MODE == M_ROWSUM || MODE == M_COLSUM) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float sA = 0.f, sB = 0.f, sC = 0.f;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const float zz = z[a][b];
          const float vA = __fmaf_rn(alA, zz, __fmaf_rn(ahA, zz, -(oA[a] + dat[b].x)));
          const float vB = __fmaf_rn(alB, zz, __fmaf_rn(ahB, zz, -(oB[a] + dat[b].z)));
          const float eA = ex2(vA);
          const float eB = ex2(vB);
          if (MODE == M_ROWSUM) {
            sA = __fmaf_rn(eA, dat[b].y, sA);
          } else {
            const float pA = eA * dat[b].y;
            sA += pA;
            sC = __fmaf_rn(zz, pA, sC);
          }
          sB = __fmaf_rn(eB, dat[b].w, sB);
        }
        ff_add(hi[a][0], lo[a][0], sA);
        ff_add(hi[a][1], lo[a][1], sB);
        if (MODE == M_COLSUM) ff_add(hi[a][NACC - 1], lo[a][NACC - 1], sC);
      }
    } else if (MODE == M_MAX) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          mx[a][0] = fmaxf(mx[a][0], __fmaf_rn(ahA, z[a][b], -dat[b].x));
          mx[a][1] = fmaxf(mx[a][1], __fmaf_rn(ahB, z[a][b], -dat[b].z));
        }
    } else if (MODE == M_MAX2) {
      // u = a z - (Rq + Bq) - Br: the offsets' sum is exact on the grid, a z exact in the fma,
      // and |u| is a few grid steps near the row maximum (Rq comes from the M_MAX pass)
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const float zz = z[a][b];
          const float u = __fmaf_rn(alA, zz, __fmaf_rn(ahA, zz, -(oA[a] + dat[b].x))) - dat[b].y;
          mx[a][0] = fmaxf(mx[a][0], u);
        }
    } else if (MODE == M_KMAX) {
      // unscaled squared distance |x|^2 + |y|^2 - 2 x.y in float32; oA holds |x_o|^2
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const bool pad = (dat[b].x == -INFINITY);
          const float dd = DIFF ? z[a][b] : __fmaf_rn(-2.0f, z[a][b], oA[a] + dat[b].x);
          mx[a][0] = fmaxf(mx[a][0], pad ? -INFINITY : dd);
          mx[a][1] = fmaxf(mx[a][1], pad ? -INFINITY : -dd);
        }
    } else if (MODE == M_GRAD) {
      // sum over inner b of 2^{v_ab} * weight_b * P_in[b][:], stream A only
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float g[DG > 0 ? DG : 1];
#pragma unroll
        for (int q = 0; q < DG; ++q) g[q] = 0.f;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const float zz = z[a][b];
          const float vA = __fmaf_rn(alA, zz, __fmaf_rn(ahA, zz, -(oA[a] + dat[b].x)));
          const float pA = ex2(vA) * dat[b].y;
          const int ib = (b < 4) ? (tx * 4 + b) : (64 + tx * 4 + b - 4);
          const float* src = Vin ? sV : sIn + q0 * kPT;
#pragma unroll
          for (int q = 0; q < DG; ++q) g[q] = __fmaf_rn(pA, src[q * kPT + ib], g[q]);
        }
#pragma unroll
        for (int q = 0; q < DG; ++q) gacc[a][q] += (double)g[q];
      }
    }
  }

  // reduce over the 16 threads (tx) that share each outer point: lanes of one half-warp
  if (MODE == M_ROWSUM || MODE == M_COLSUM) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      int64_t go = o0 + ((a < 4) ? (ty * 4 + a) : (64 + ty * 4 + a - 4));
#pragma unroll
      for (int q = 0; q < NACC; ++q) {
        double v = (double)hi[a][q] + (double)lo[a][q];
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (tx == 0 && go < n_out) part[((int64_t)split * NACC + q) * n_out + go] = v;
      }
    }
  } else if (MODE == M_MAX || MODE == M_KMAX || MODE == M_MAX2) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      int64_t go = o0 + ((a < 4) ? (ty * 4 + a) : (64 + ty * 4 + a - 4));
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float v = mx[a][q];
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (tx == 0 && go < n_out) pmax[((int64_t)split * 2 + q) * n_out + go] = v;
      }
    }
  } else if (MODE == M_GRAD) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      int64_t go = o0 + ((a < 4) ? (ty * 4 + a) : (64 + ty * 4 + a - 4));
#pragma unroll
      for (int q = 0; q < DG; ++q) {
        double v = gacc[a][q];
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (tx == 0 && go < n_out) part[((int64_t)split * n_out + go) * DG + q] = v;
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// sweeps over a stored dense cost (LAMP_COST_DENSE), streamed from HBM with coalesced loads

constexpr int kDR = 8;        // rows per CTA in the row sweep
constexpr int kDChunk = 1024; // columns per CTA step (4 per thread, stride 256)

template <int MODE>  // M_ROWSUM, M_MAX or M_MAX2
__global__ void __launch_bounds__(kThreads)
k_dense_rows(const float* __restrict__ C, int64_t ldc, int64_t n, int64_t m, const Work w,
             int chunks_per_split, const Consts k) {
  const DevState* __restrict__ dev = w.dev;
  if (MODE == M_ROWSUM && dev->done) return;
  const int cur = dev->cur;
  const float2* __restrict__ rowshift = w.rowshift[cur];
  const float4* __restrict__ colq = w.colq[cur];
  double* __restrict__ part = w.rowpart;
  float* __restrict__ pmax = w.rowmax;
  __shared__ double sred[kThreads / 32][kDR * 2];
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kDR;
  const int split = blockIdx.y;
  const int64_t nchunks = (m + kDChunk - 1) / kDChunk;
  const int64_t c0 = (int64_t)split * chunks_per_split;
  int64_t c1 = c0 + chunks_per_split;
  if (c1 > nchunks) c1 = nchunks;
  const SweepF sp = sweep_floats_of(dev, k);
  const float ahA = sp.ahA, alA = sp.alA, ahB = sp.ahB, alB = sp.alB;

  float oA[kDR], oB[kDR];
  const float* crow[kDR];
#pragma unroll
  for (int a = 0; a < kDR; ++a) {
    int64_t gr = r0 + a;
    if (gr >= n) gr = n - 1;
    float2 q = MODE == M_MAX ? make_float2(0.f, 0.f) : rowshift[gr];
    oA[a] = q.x;
    oB[a] = q.y;
    crow[a] = C + gr * ldc;
  }
  float hiA[kDR], loA[kDR], hiB[kDR], loB[kDR];
  float mA[kDR], mB[kDR];
#pragma unroll
  for (int a = 0; a < kDR; ++a) {
    hiA[a] = loA[a] = hiB[a] = loB[a] = 0.f;
    mA[a] = mB[a] = -INFINITY;
  }

  for (int64_t ch = c0; ch < c1; ++ch) {
    float4 cd[4];
    int64_t jj[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      jj[q] = ch * kDChunk + tid + q * kThreads;
      cd[q] = jj[q] < m ? colq[jj[q]] : make_float4(INFINITY, 0.f, INFINITY, 0.f);
    }
    float cv[kDR][4];
#pragma unroll
    for (int a = 0; a < kDR; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) cv[a][q] = jj[q] < m ? __ldg(crow[a] + jj[q]) : 0.f;
#pragma unroll
    for (int a = 0; a < kDR; ++a) {
      if (MODE == M_ROWSUM) {
        float sA = 0.f, sB = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float zz = cv[a][q];
          const float vA = __fmaf_rn(alA, zz, __fmaf_rn(ahA, zz, -(oA[a] + cd[q].x)));
          const float vB = __fmaf_rn(alB, zz, __fmaf_rn(ahB, zz, -(oB[a] + cd[q].z)));
          sA = __fmaf_rn(ex2(vA), cd[q].y, sA);
          sB = __fmaf_rn(ex2(vB), cd[q].w, sB);
        }
        ff_add(hiA[a], loA[a], sA);
        ff_add(hiB[a], loB[a], sB);
      } else if (MODE == M_MAX2) {
        // refinement pass of the eta = 0 dual bound (see k_pts_sweep, M_MAX2)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float zz = cv[a][q];
          mA[a] = fmaxf(mA[a], __fmaf_rn(alA, zz, __fmaf_rn(ahA, zz, -(oA[a] + cd[q].x))) - cd[q].y);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          mA[a] = fmaxf(mA[a], __fmaf_rn(ahA, cv[a][q], -cd[q].x));
          mB[a] = fmaxf(mB[a], __fmaf_rn(ahB, cv[a][q], -cd[q].z));
        }
      }
    }
  }

  const int lane = tid & 31, wid = tid >> 5;
  if (MODE == M_ROWSUM) {
#pragma unroll
    for (int a = 0; a < kDR; ++a) {
      warp_sum_ff(hiA[a], loA[a]);
      warp_sum_ff(hiB[a], loB[a]);
      const double vA = (double)hiA[a] + (double)loA[a];
      const double vB = (double)hiB[a] + (double)loB[a];
      if (lane == 0) {
        sred[wid][2 * a] = vA;
        sred[wid][2 * a + 1] = vB;
      }
    }
    __syncthreads();
    if (tid < 2 * kDR) {
      double v = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) v += sred[w][tid];
      int a = tid >> 1, s = tid & 1;
      if (r0 + a < n) part[((int64_t)split * 2 + s) * n + r0 + a] = v;
    }
  } else {
    __shared__ float fred[kThreads / 32][kDR * 2];
#pragma unroll
    for (int a = 0; a < kDR; ++a) {
      float vA = warp_max_f(mA[a]);
      float vB = warp_max_f(mB[a]);
      if (lane == 0) {
        fred[wid][2 * a] = vA;
        fred[wid][2 * a + 1] = vB;
      }
    }
    __syncthreads();
    if (tid < 2 * kDR) {
      float v = -INFINITY;
      for (int w = 0; w < kThreads / 32; ++w) v = fmaxf(v, fred[w][tid]);
      int a = tid >> 1, s = tid & 1;
      if (r0 + a < n) pmax[((int64_t)split * 2 + s) * n + r0 + a] = v;
    }
  }
}

constexpr int kDColRows = 16;  // rows per step (row data staged in shared memory)

__global__ void __launch_bounds__(kThreads)
k_dense_cols(const float* __restrict__ C, int64_t ldc, int64_t n, int64_t m, const Work w, int64_t rows_per_split,
             const Consts k) {
  const DevState* __restrict__ dev = w.dev;
  if (dev->done) return;
  const float4* __restrict__ g2row = w.g2row;
  const float4* __restrict__ colq = w.colq[dev->cur];
  double* __restrict__ part = w.colpart;
  __shared__ float4 srow[kDColRows];
  const int tid = threadIdx.x;
  const int64_t jb = (int64_t)blockIdx.x * kDChunk;
  const int split = blockIdx.y;
  const int64_t i0 = (int64_t)split * rows_per_split;
  int64_t i1 = i0 + rows_per_split;
  if (i1 > n) i1 = n;
  const SweepF sp = sweep_floats_of(dev, k);
  const float ahA = sp.ahA, alA = sp.alA, ahB = sp.ahB, alB = sp.alB;

  float oA[4], oB[4];
  int64_t jj[4];
  bool ok[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    jj[q] = jb + tid + q * kThreads;
    ok[q] = jj[q] < m;
    float4 cd = ok[q] ? colq[jj[q]] : make_float4(0.f, 0.f, 0.f, 0.f);
    oA[q] = cd.x;
    oB[q] = cd.z;
  }
  float hiA[4], loA[4], hiB[4], loB[4], hiC[4], loC[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) hiA[q] = loA[q] = hiB[q] = loB[q] = hiC[q] = loC[q] = 0.f;

  for (int64_t ib = i0; ib < i1; ib += kDColRows) {
    __syncthreads();
    if (tid < kDColRows) {
      int64_t gi = ib + tid;
      srow[tid] = gi < i1 ? g2row[gi] : make_float4(INFINITY, 0.f, INFINITY, 0.f);
    }
    __syncthreads();
    float sA[4] = {0.f, 0.f, 0.f, 0.f}, sB[4] = {0.f, 0.f, 0.f, 0.f}, sC[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int a = 0; a < kDColRows; ++a) {
      int64_t gi = ib + a;
      if (gi >= i1) break;
      const float4 rd = srow[a];
      const float* crow = C + gi * ldc;
      float cv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) cv[q] = ok[q] ? __ldg(crow + jj[q]) : 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float zz = cv[q];
        const float vA = __fmaf_rn(alA, zz, __fmaf_rn(ahA, zz, -(oA[q] + rd.x)));
        const float vB = __fmaf_rn(alB, zz, __fmaf_rn(ahB, zz, -(oB[q] + rd.z)));
        const float pA = ex2(vA) * rd.y;
        sA[q] += pA;
        sC[q] = __fmaf_rn(zz, pA, sC[q]);
        sB[q] = __fmaf_rn(ex2(vB), rd.w, sB[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ff_add(hiA[q], loA[q], sA[q]);
      ff_add(hiB[q], loB[q], sB[q]);
      ff_add(hiC[q], loC[q], sC[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!ok[q]) continue;
    part[((int64_t)split * 3 + 0) * m + jj[q]] = (double)hiA[q] + (double)loA[q];
    part[((int64_t)split * 3 + 1) * m + jj[q]] = (double)hiB[q] + (double)loB[q];
    part[((int64_t)split * 3 + 2) * m + jj[q]] = (double)hiC[q] + (double)loC[q];
  }
}

// dense cost: max, min and finiteness of C (the K pass, Section 2: K = ||C||_inf)
__global__ void k_dense_stats(const float* __restrict__ C, int64_t ldc, int64_t n, int64_t m, double* out) {
  __shared__ float smx[kThreads / 32], smn[kThreads / 32];
  __shared__ int sbad[kThreads / 32];
  float mx = -INFINITY, mn = INFINITY;
  int bad = 0;
  const int64_t total = n * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / m, j = e - i * m;
    float v = C[i * ldc + j];
    if (!isfinite(v)) bad = 1;
    mx = fmaxf(mx, v);
    mn = fminf(mn, v);
  }
  mx = warp_max_f(mx);
  mn = warp_min_f(mn);
  bad = __any_sync(0xffffffffu, bad);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { smx[wid] = mx; smn[wid] = mn; sbad[wid] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) { mx = fmaxf(mx, smx[w]); mn = fminf(mn, smn[w]); bad |= sbad[w]; }
    mx = fmaxf(mx, smx[0]); mn = fminf(mn, smn[0]); bad |= sbad[0];
    out[3 * blockIdx.x + 0] = mx;
    out[3 * blockIdx.x + 1] = mn;
    out[3 * blockIdx.x + 2] = bad;
  }
}

// ------------------------------------------------------------------------------------------
// O(n + m) kernels

__global__ void k_norms(const float* __restrict__ P, int64_t np, int d, double* __restrict__ nrm,
                        float2* __restrict__ f2, float4* __restrict__ f4) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  double s = 0.0;
  float sf = 0.f;
  for (int k = 0; k < d; ++k) {
    float v = P[i * d + k];
    s += (double)v * (double)v;
    sf = __fmaf_rn(v, v, sf);
  }
  nrm[i] = s;
  if (f2) f2[i] = make_float2(sf, 0.f);
  if (f4) f4[i] = make_float4(sf, 0.f, 0.f, 0.f);
}

// cosine cost: out_i = P_i / (sqrt 2 |P_i|) (float64 norm); rows with a zero or non-finite
// norm are counted in *bad and written as zeros
__global__ void k_unit_rows(const float* __restrict__ P, int64_t np, int d, float* __restrict__ out,
                            unsigned int* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  double s = 0.0;
  for (int q = 0; q < d; ++q) s += (double)P[i * d + q] * (double)P[i * d + q];
  double sc = 0.0;
  if (s > 0.0 && isfinite(s)) sc = 1.0 / sqrt(2.0 * s);
  else atomicAdd(bad, 1u);
  for (int q = 0; q < d; ++q) out[i * d + q] = (float)((double)P[i * d + q] * sc);
}

// marginal checks: sum, min, finiteness (block partials, 3 doubles per block)
__global__ void k_vec_stats(const double* __restrict__ v, int64_t len, double* out) {
  __shared__ double ssum[kThreads / 32], smn[kThreads / 32], sbad[kThreads / 32];
  double s = 0.0, mn = INFINITY, bad = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    double x = v[i];
    if (!isfinite(x)) bad = 1.0;
    s += x;
    mn = fmin(mn, x);
  }
  s = warp_sum_d(s);
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    bad = fmax(bad, __shfl_xor_sync(0xffffffffu, bad, o));
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { ssum[wid] = s; smn[wid] = mn; sbad[wid] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, M = INFINITY, B = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) { S += ssum[w]; M = fmin(M, smn[w]); B = fmax(B, sbad[w]); }
    out[3 * blockIdx.x + 0] = S;
    out[3 * blockIdx.x + 1] = M;
    out[3 * blockIdx.x + 2] = B;
  }
}

// set the column data of the current state buffer from its (nu, theta) and dev->kappa
__global__ void k_init_cols(const Work w, const Consts k, int zero) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k.m) return;
  const DevState* __restrict__ dev = w.dev;
  const int cur = dev->cur;
  const double* __restrict__ ny = w.ny;
  double* __restrict__ nu = w.nu[cur];
  double* __restrict__ theta = w.theta[cur];
  float4* __restrict__ colq = w.colq[cur];
  if (zero) { nu[j] = 0.0; theta[j] = 0.0; }
  SweepParams sp = make_sweep_params(sweep_kappa(dev->kappa, k), k);
  double wt = k.tau1 / sp.kapB;  // tau1 eta_{t+1}
  double nb = nu[j] + wt * (theta[j] - nu[j]);
  double sny = k.zdot ? k.s * ny[j] : 0.0;
  float dB;
  const float4 cd = column_data(nu[j], nb, sny, sp, k, &dB);
  colq[j] = cd;
  if (w.colq2[cur]) store_pair_entry(w.colq2[cur], j, cd.x, cd.y, dB, cd.w);
}

// row shifts from the prime pass' row maxima: Rq = round_g(max_j (a z_ij - Bq_j))
__global__ void k_prime_fin(const Work w, int splits, const Consts k) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k.n) return;
  const DevState* __restrict__ dev = w.dev;
  const float* __restrict__ pmax = w.rowmax;
  float2* __restrict__ rowshift = w.rowshift[dev->cur];
  SweepParams sp = make_sweep_params(sweep_kappa(dev->kappa, k), k);
  float mA = -INFINITY, mB = -INFINITY;
  for (int s = 0; s < splits; ++s) {
    mA = fmaxf(mA, pmax[((int64_t)s * 2 + 0) * k.n + i]);
    mB = fmaxf(mB, pmax[((int64_t)s * 2 + 1) * k.n + i]);
  }
  double qA = isfinite(mA) ? quantize((double)mA, sp.g) : 0.0;
  double qB = isfinite(mB) ? quantize((double)mB, sp.g) : 0.0;
  if (k.shared_shift) qB = qA;
  rowshift[i] = make_float2((float)qA, (float)qB);
}

// RF: row finalize of iteration t
__global__ void __launch_bounds__(kFinThreads)
k_row_fin(const Work w, int splits, const double* __restrict__ r, const Consts k) {
  DevState* __restrict__ dev = w.dev;
  if (dev->done) return;
  const int cur = dev->cur;
  const double* __restrict__ rowpart = w.rowpart;
  const double* __restrict__ nx = w.nx;
  const float2* __restrict__ rs_cur = w.rowshift[cur];
  float2* __restrict__ rs_nxt = w.rowshift[cur ^ 1];
  float4* __restrict__ g2row = w.g2row;
  double* __restrict__ logZ = w.logZ;
  double* __restrict__ rowred = w.rowred;
  __shared__ double sred[kFinThreads / 32];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (i < k.n) {
    SweepParams sp, spn;
    iteration_params_of(dev, k, sp, spn);
    double SA = 0.0, SB = 0.0;
    // unrolled: the partials' loads are independent and in flight together; the sums keep
    // the split order
#pragma unroll 8
    for (int s = 0; s < splits; ++s) {
      SA += rowpart[((int64_t)s * 2 + 0) * k.n + i];
      SB += rowpart[((int64_t)s * 2 + 1) * k.n + i];
    }
    const double lim = 1.0e36;
    if (!(SA > 1.0 / lim && SA < lim && SB > 1.0 / lim && SB < lim)) {
      atomicExch(&dev->status, 5 /* LAMP_E_NUMERIC */);
      SA = SA > 0 ? SA : 1.0;
      SB = SB > 0 ? SB : 1.0;
    }
    float2 rq = rs_cur[i];
    double snx = k.zdot ? k.s * nx[i] : 0.0;
    // float64 log2 and divisions: with float32 ones (log2f carries an absolute error of
    // ~2^-22 near 1) the potentials of 100-iteration trajectories drifted from the oracle's
    // by ~1e-6 instead of ~1e-8, and log Z, which amplifies nu by 2 K kappa, by ~1e-4
    const double lsA = log2(SA), lsB = log2(SB);
    double L2A = (double)rq.x - sp.lamA * snx + lsA;  // log2 Z of X^t
    double L2B = (double)rq.y - sp.lamB * snx + lsB;  // log2 Z of Xbar^{t+1}
    double lz = kLn2 * L2A;
    logZ[i] = lz;
    double ri = r[i];
    contrib = ri * lz;
    // the row weights q = r / S, float32 factors of the column sweep
    const float qa = (float)(ri / SA), qb = (float)(ri / SB);
    g2row[i] = make_float4(rq.x, qa, rq.y, qb);
    if (w.g2row2) store_pair_entry(w.g2row2, i, rq.x, qa, 0.f, qb);
    // shifts of iteration t+1: stream A there has kappa_{t+1} (stream B here);
    // stream B there is extrapolated linearly in t.
    double tA = (double)rq.y + lsB;
    double tB = spn.lamB * snx + 2.0 * L2B - L2A;
    const float qA = (float)quantize(tA, spn.g);
    rs_nxt[i] = make_float2(qA, k.shared_shift ? qA : (float)quantize(tB, spn.g));
  }
  contrib = warp_sum_d(contrib);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sred[wid] = contrib;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kFinThreads / 32; ++w) v += sred[w];
    rowred[blockIdx.x] = v;
  }
}

// CF: column finalize of iteration t, dual step of Alg. 2, and the decision
__global__ void __launch_bounds__(kFinThreads)
k_col_fin(const Work w, int splits, const double* __restrict__ cvec, int rowblocks, int with_cost, const Consts k) {
  DevState* __restrict__ dev = w.dev;
  if (dev->done) return;
  const int cur = dev->cur;
  const double* __restrict__ colpart = w.colpart;
  const double* __restrict__ ny = w.ny;
  const float4* __restrict__ colq_cur = w.colq[cur];
  float4* __restrict__ colq_nxt = w.colq[cur ^ 1];
  const double* __restrict__ nu_cur = w.nu[cur];
  const double* __restrict__ th_cur = w.theta[cur];
  double* __restrict__ nu_nxt = w.nu[cur ^ 1];
  double* __restrict__ th_nxt = w.theta[cur ^ 1];
  double* __restrict__ colA = w.colA;
  double* __restrict__ colred = w.colred;
  const double* __restrict__ rowred = w.rowred;
  __shared__ double sred[4][kFinThreads / 32];
  __shared__ bool amLast;
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double res = 0.0, cost = 0.0, cnu = 0.0;
  SweepParams sp, spn;
  iteration_params_of(dev, k, sp, spn);
  const int eval_only = dev->eval_only;
  if (j < k.m) {
    double aA = 0.0, aB = 0.0, aC = 0.0;
    // partials of split s: [s][3][m] with the cost-weighted sums, [s][2][m] without
    const int na = with_cost ? 3 : 2;
    // unrolled: the partials' loads are independent and in flight together; the sums keep
    // the split order
#pragma unroll 8
    for (int s = 0; s < splits; ++s) {
      aA += colpart[((int64_t)s * na + 0) * k.m + j];
      aB += colpart[((int64_t)s * na + 1) * k.m + j];
      if (with_cost) aC += colpart[((int64_t)s * na + 2) * k.m + j];
    }
    float4 cq = colq_cur[j];
    const double A = (double)cq.y * aA;  // col(X^t)_j
    // col(Xbar^{t+1})_j; under the shared row shift the column weight of stream B is
    // already inside the sweep's exponents
    const double B = k.shared_shift ? aB : (double)cq.w * aB;
    const double zsum = (double)cq.y * aC;
    if (!k.zdot) {
      cost = k.s * zsum;
    } else {
      cost = k.s * ny[j] * A - 2.0 * k.s * zsum;  // + sum_i r_i s|x_i|^2 added once below
    }
    const double cj = cvec[j];
    const double nuj = nu_cur[j], thj = th_cur[j];
    res = fabs(A - cj);
    cnu = A * nuj;
    colA[j] = A;
    if (with_cost && w.colz) w.colz[j] = cost;
    if (!eval_only) {
      // the dual mirror steps (Eq. def:closed_form_opt) tanh(g (col - c) + atanh theta), in
      // float64 through the addition theorem tanh(u + atanh theta) = (tanh u + theta) /
      // (1 + theta tanh u): one tanh per stream and no atanh (|theta^t| <= tanh(beta/2) < 1,
      // so the denominator is at least 1 - tanh(beta/2))
      const double ca = cj + k.alpha_m;                  // c^alpha (Section 3.1)
      const double gj = 2.0 * k.tau2 * k.K / ca;
      const double wt = sp.wB;                           // tau1 eta_{t+1}
      const double tA = tanh(gj * (A - cj));
      const double thbar = (tA + thj) / fma(tA, thj, 1.0);  // M_{tau2}(theta^t; p^{eta_t}(nu^t))
      const double nun = nuj + wt * (thbar - nuj);       // nu^{t+1}
      const double tB = tanh(gj * (B - cj));
      const double thhat = (tB + thj) / fma(tB, thj, 1.0);  // M_{tau2}(theta^t; p^{eta_{t+1}}(nubar^{t+1}))
      const double thn = fmin(fmax(thhat, -k.clipb), k.clipb);  // tclip
      nu_nxt[j] = nun;
      th_nxt[j] = thn;
      // column data of iteration t+1
      const double wn = spn.wB;
      const double nbn = nun + wn * (thn - nun);         // nubar^{t+2}
      const double sny = k.zdot ? k.s * ny[j] : 0.0;
      float dB;
      const float4 cd = column_data(nun, nbn, sny, spn, k, &dB);
      colq_nxt[j] = cd;
      if (w.colq2[cur ^ 1]) store_pair_entry(w.colq2[cur ^ 1], j, cd.x, cd.y, dB, cd.w);
    }
  }
  res = warp_sum_d(res);
  cost = warp_sum_d(cost);
  cnu = warp_sum_d(cnu);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sred[0][wid] = res; sred[1][wid] = cost; sred[2][wid] = cnu; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int w = 0; w < kFinThreads / 32; ++w) { a += sred[0][w]; b += sred[1][w]; c += sred[2][w]; }
    colred[3 * blockIdx.x + 0] = a;
    colred[3 * blockIdx.x + 1] = b;
    colred[3 * blockIdx.x + 2] = c;
    __threadfence();
    unsigned int tk = atomicAdd(&dev->ticket, 1u);
    amLast = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!amLast) return;
  // last block: reduce all partials in a fixed order (thread t takes blocks t, t + 128, ..,
  // then a fixed tree over the threads) and decide
  __threadfence();
  double R = 0.0, Cx = 0.0, Cn = 0.0, RL = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    R += ((volatile double*)colred)[3 * b + 0];
    Cx += ((volatile double*)colred)[3 * b + 1];
    Cn += ((volatile double*)colred)[3 * b + 2];
  }
  for (int b = threadIdx.x; b < rowblocks; b += blockDim.x) RL += ((volatile const double*)rowred)[b];
  R = warp_sum_d(R);
  Cx = warp_sum_d(Cx);
  Cn = warp_sum_d(Cn);
  RL = warp_sum_d(RL);
  __syncthreads();  // sred is reused
  if (lane == 0) { sred[0][wid] = R; sred[1][wid] = Cx; sred[2][wid] = Cn; sred[3][wid] = RL; }
  __syncthreads();
  if (threadIdx.x == 0) {
    R = Cx = Cn = RL = 0.0;
    for (int w = 0; w < kFinThreads / 32; ++w) { R += sred[0][w]; Cx += sred[1][w]; Cn += sred[2][w]; RL += sred[3][w]; }
    Cx += k.rnx;
    dev->ticket = 0u;
    dev->res = R;
    dev->costA = with_cost ? Cx : NAN;
    dev->colnu = Cn;
    dev->rlogZ = RL;
    dev->t_eval = dev->t;
    dev->kappa_eval = dev->kappa;
    if (dev->status != 0 || !isfinite(R)) {
      if (dev->status == 0) dev->status = 5;
      dev->done = 1;
    } else if (eval_only) {
      dev->done = 1;
    } else if ((dev->t >= 1 && R <= dev->tol &&
                (k.eta == 0.0 || k.infeas_only || 1.0 - dev->kappa * k.eta <= dev->tol)) ||
               dev->t >= dev->tmax) {
      dev->done = 1;
    } else {
      dev->t = dev->t + 1;
      dev->kappa = sp.kapB;
      dev->cur ^= 1;
      if (k.kap_ovr < 0.0 && !k.same_kappa) {
        // the next iteration's parameters, once per iteration instead of once per thread
        // (float64 is slow on this part)
        dev->spc = spn;
        dev->spn = make_sweep_params(spn.kapB, k);
        dev->swf = sweep_floats(spn);
        dev->swf_kap = spn.kapA;
      }
    }
    __threadfence();
  }
}

// gradient finalize of coordinates q0 .. q0 + dg - 1 (partials hold dg values per point):
// dx_i = 2 s (r_i x_i - q_i acc_i)
__global__ void k_grad_fin(const double* __restrict__ part, int splits, int64_t np, int dg, int q0, int d,
                           const float* __restrict__ P, const double* __restrict__ mass,
                           const float4* __restrict__ wsrc, int wcomp, double s, float* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  float4 wq = wsrc[i];
  double wgt = (double)(wcomp == 1 ? wq.y : wq.w);
  double ms = mass[i];
  for (int q = 0; q < dg; ++q) {
    double acc = 0.0;
    for (int sp = 0; sp < splits; ++sp) acc += part[((int64_t)sp * np + i) * dg + q];
    out[i * d + q0 + q] = (float)(2.0 * s * (ms * (double)P[i * d + q0 + q] - wgt * acc));
  }
}

// column gradient finalize of coordinates q0 .. q0 + dg - 1: dy_j = 2 s (A_j y_j - w_j acc_j),
// w_j from the current column data
__global__ void k_grad_fin_cols(const Work w, int splits, int64_t np, int dg, int q0, int d,
                                const float* __restrict__ P, double s, float* __restrict__ out) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  float4 cq = w.colq[w.dev->cur][j];
  double wgt = (double)cq.y;
  double ms = w.colA[j];
  for (int q = 0; q < dg; ++q) {
    double acc = 0.0;
    for (int sp = 0; sp < splits; ++sp) acc += w.colpart[((int64_t)sp * np + j) * dg + q];
    out[j * d + q0 + q] = (float)(2.0 * s * (ms * (double)P[j * d + q0 + q] - wgt * acc));
  }
}

// ------------------------------------------------------------------------------------------
// launch glue

static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

static size_t pts_smem(int d, int dv = 0) {
  return (size_t)(2 * d * kPT + dv * kPT) * sizeof(float) + kPT * sizeof(float4);
}

static SweepIO io_same(const float2* o2, const float4* o4, const float4* in) {
  SweepIO io;
  io.off2[0] = io.off2[1] = o2;
  io.off4[0] = io.off4[1] = o4;
  io.indat[0] = io.indat[1] = in;
  return io;
}

template <int MODE, int DG>
static cudaError_t launch_pts(const float* Pout, const float* Pin, int64_t nout, int64_t nin, int d, const SweepIO& io,
                              double* part, float* pmax, int splits, const DevState* dev, const Consts& k,
                              cudaStream_t st, const float* V = nullptr, int q0 = 0) {
  auto kern = k.zdot ? k_pts_sweep<MODE, DG, false> : k_pts_sweep<MODE, DG, true>;
  size_t sm = pts_smem(d, V ? DG : 0);
  int64_t tin = cdiv(nin, kPT);
  int tps = (int)cdiv(tin, splits);
  dim3 grid((unsigned)cdiv(nout, kPT), (unsigned)splits);
  kern<<<grid, kThreads, sm, st>>>(Pout, Pin, nout, nin, d, io, part, pmax, tps, dev, k, V, q0);
  return cudaGetLastError();
}

// the packed direct-form sweeps serve |x - y|^2 with d <= 8 in float32
bool uses_direct_sweeps(const Consts& k, int prec) {
  return k.kind == COST_SQEUCLID && !k.zdot && prec != 1 /* LAMP_PREC_BF16_TC */ && k.d >= 1 && k.d <= 8;
}

cudaError_t launch_unit_rows(const float* P, int64_t np, int d, float* out, unsigned int* bad, cudaStream_t st) {
  k_unit_rows<<<(unsigned)cdiv(np, 256), 256, 0, st>>>(P, np, d, out, bad);
  return cudaGetLastError();
}

cudaError_t launch_norms(const Inputs& in, const Consts& k, const Work& w, cudaStream_t st) {
  if (k.kind != COST_SQEUCLID) return cudaSuccess;
  // float32 norms go into buffers that are unused before the first iteration
  k_norms<<<(unsigned)cdiv(k.n, 256), 256, 0, st>>>(in.x, k.n, k.d, w.nx, w.rowshift[1], nullptr);
  k_norms<<<(unsigned)cdiv(k.m, 256), 256, 0, st>>>(in.y, k.m, k.d, w.ny, nullptr, w.colq[1]);
  return cudaGetLastError();
}

// the K pass's column data in the packed-pair layout: -offA = |y_j|^2 (the float norms that
// k_norms left in f4[j].x)
__global__ void k_norm_pairs(const float4* __restrict__ f4, float4* __restrict__ pairs, int64_t m) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) store_pair_entry(pairs, j, -f4[j].x, 0.f, 0.f, 0.f);
}

cudaError_t launch_kmax(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                        cudaStream_t st) {
  if (k.kind == COST_DENSE) {
    k_dense_stats<<<4 * g.sms, kThreads, 0, st>>>(in.C, in.ldc, k.n, k.m, w.scratch);
    return cudaGetLastError();
  }
  if (prec == 1 /* LAMP_PREC_BF16_TC */ && g.map_x && w.colq2[1]) {
    // on the tensor cores, with the products of the bf16 points the iteration uses: the
    // row data (rowshift[1].x) hold |x_i|^2, the pair data |y_j|^2
    k_norm_pairs<<<(unsigned)cdiv(k.m, 256), 256, 0, st>>>(w.colq[1], w.colq2[1], k.m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    Work w2 = w;
    w2.rowshift[0] = w2.rowshift[1] = w.rowshift[1];
    w2.colq2[0] = w2.colq2[1] = w.colq2[1];
    return tc_launch_rowmax(3, g, w2, k, g.rows_split, st);
  }
  // rowmax[split][0][n] = max_j D_ij, rowmax[split][1][n] = max_j -D_ij, D = |x|^2 + |y|^2 - 2 x.y
  return launch_pts<M_KMAX, 0>(in.x, in.y, k.n, k.m, k.d, io_same(w.rowshift[1], nullptr, w.colq[1]), nullptr,
                               w.rowmax, g.rows_split, w.dev, k, st);
}

cudaError_t launch_check_marginals(const Inputs& in, const Consts& k, const Work& w, cudaStream_t st) {
  k_vec_stats<<<64, kThreads, 0, st>>>(in.r, k.n, w.scratch);
  k_vec_stats<<<64, kThreads, 0, st>>>(in.c, k.m, w.scratch + 3 * 64);
  return cudaGetLastError();
}

cudaError_t launch_init_state(const Inputs& in, const Consts& k, const Work& w, int zero, cudaStream_t st) {
  k_init_cols<<<(unsigned)cdiv(k.m, 256), 256, 0, st>>>(w, k, zero);
  return cudaGetLastError();
}

static cudaError_t launch_row_sweep(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int mode,
                                    cudaStream_t st) {
  if (k.kind == COST_DENSE && g.map_c && mode == M_ROWSUM) return dense_launch_sweep(true, 0, g, w, k, g.rows_split, st);
  if (k.kind == COST_DENSE) {
    int64_t nch = cdiv(k.m, kDChunk);
    int cps = (int)cdiv(nch, g.rows_split);
    dim3 grid((unsigned)cdiv(k.n, kDR), (unsigned)g.rows_split);
    if (mode == M_ROWSUM)
      k_dense_rows<M_ROWSUM><<<grid, kThreads, 0, st>>>(in.C, in.ldc, k.n, k.m, w, cps, k);
    else if (mode == M_MAX2)
      k_dense_rows<M_MAX2><<<grid, kThreads, 0, st>>>(in.C, in.ldc, k.n, k.m, w, cps, k);
    else
      k_dense_rows<M_MAX><<<grid, kThreads, 0, st>>>(in.C, in.ldc, k.n, k.m, w, cps, k);
    return cudaGetLastError();
  }
  if (mode == M_ROWSUM && k.shared_shift) return launch_direct_sweep(true, 0, in, k, w, g, st);
  SweepIO io;
  for (int b = 0; b < 2; ++b) {
    io.off2[b] = w.rowshift[b];
    io.off4[b] = nullptr;
    io.indat[b] = w.colq[b];
  }
  if (mode == M_ROWSUM)
    return launch_pts<M_ROWSUM, 0>(in.x, in.y, k.n, k.m, k.d, io, w.rowpart, nullptr, g.rows_split, w.dev, k, st);
  if (mode == M_MAX2)
    return launch_pts<M_MAX2, 0>(in.x, in.y, k.n, k.m, k.d, io, nullptr, w.rowmax, g.rows_split, w.dev, k, st);
  return launch_pts<M_MAX, 0>(in.x, in.y, k.n, k.m, k.d, io, nullptr, w.rowmax, g.rows_split, w.dev, k, st);
}

static cudaError_t launch_col_sweep(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int eval,
                                    cudaStream_t st) {
  // stored costs accumulate <C, X^t> in every iteration (the column finalize reads three
  // partials per split whenever the row shift is not shared)
  if (k.kind == COST_DENSE && g.map_c) return dense_launch_sweep(false, 1, g, w, k, g.cols_split, st);
  if (k.kind == COST_DENSE) {
    int64_t rps = cdiv(k.n, g.cols_split);
    rps = cdiv(rps, kDColRows) * kDColRows;
    dim3 grid((unsigned)cdiv(k.m, kDChunk), (unsigned)g.cols_split);
    k_dense_cols<<<grid, kThreads, 0, st>>>(in.C, in.ldc, k.n, k.m, w, rps, k);
    return cudaGetLastError();
  }
  if (k.shared_shift) return launch_direct_sweep(false, eval, in, k, w, g, st);
  SweepIO io;
  for (int b = 0; b < 2; ++b) {
    io.off2[b] = nullptr;
    io.off4[b] = w.colq[b];
    io.indat[b] = w.g2row;
  }
  return launch_pts<M_COLSUM, 0>(in.y, in.x, k.m, k.n, k.d, io, w.colpart, nullptr, g.cols_split, w.dev, k, st);
}

cudaError_t launch_prime(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                         cudaStream_t st) {
  // the tensor-core context takes its row maxima from the tensor-core sweep (the cost its
  // iteration uses)
  cudaError_t e = prec == 1 /* LAMP_PREC_BF16_TC */ && g.map_x ? tc_launch_rowmax(1, g, w, k, g.rows_split, st)
                                                                : launch_row_sweep(in, k, w, g, M_MAX, st);
  if (e != cudaSuccess) return e;
  k_prime_fin<<<(unsigned)cdiv(k.n, 256), 256, 0, st>>>(w, g.rows_split, k);
  return cudaGetLastError();
}

cudaError_t launch_rowmax_refined(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                                  cudaStream_t st) {
  if (prec == 1 /* LAMP_PREC_BF16_TC */ && g.map_x) return tc_launch_rowmax(2, g, w, k, g.rows_split, st);
  return launch_row_sweep(in, k, w, g, M_MAX2, st);
}

cudaError_t launch_iteration_part(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                                  int part, int eval, cudaStream_t st) {
  const int rb = (int)fin_blocks(k.n);
  const bool tcpath = prec == 1 /* LAMP_PREC_BF16_TC */;
  switch (part) {
    case 0:
      if (tcpath) return tc_launch_sweep(true, 0, g, w, k, g.rows_split, st);
      return launch_row_sweep(in, k, w, g, M_ROWSUM, st);
    case 1:
      k_row_fin<<<rb, kFinThreads, 0, st>>>(w, g.rows_split, in.r, k);
      return cudaGetLastError();
    case 2:
      if (tcpath) return tc_launch_sweep(false, eval, g, w, k, g.cols_split, st);
      return launch_col_sweep(in, k, w, g, eval, st);
    default:
      // the packed direct-form column sweep accumulates <C, X> in evaluation passes only
      k_col_fin<<<(unsigned)fin_blocks(k.m), kFinThreads, 0, st>>>(w, g.cols_split, in.c, rb,
                                                                    eval || !k.shared_shift, k);
      return cudaGetLastError();
  }
}

cudaError_t launch_iteration(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                             int eval, cudaStream_t st) {
  for (int part = 0; part < 4; ++part) {
    cudaError_t e = launch_iteration_part(in, k, w, g, prec, part, eval, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int launches_per_iteration(const Consts& k, int prec) { return 4; }

template <int MODE, int DG>
static void set_attr() {
  const int sm = (int)pts_smem(64, DG);
  cudaFuncSetAttribute(k_pts_sweep<MODE, DG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_pts_sweep<MODE, DG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

// raise the dynamic shared-memory limit of every sweep instantiation once, before any capture
void prepare_kernels() {
  static bool done = false;
  if (done) return;
  set_attr<M_ROWSUM, 0>();
  set_attr<M_COLSUM, 0>();
  set_attr<M_MAX, 0>();
  set_attr<M_MAX2, 0>();
  set_attr<M_KMAX, 0>();
  set_attr<M_GRAD, 1>();
  set_attr<M_GRAD, 2>();
  set_attr<M_GRAD, 3>();
  set_attr<M_GRAD, 4>();
  set_attr<M_GRAD, 5>();
  set_attr<M_GRAD, 6>();
  set_attr<M_GRAD, 7>();
  set_attr<M_GRAD, 8>();
  done = true;
}

int sweep_blocks_per_sm(const Consts& k, int prec, int which) {
  int nb = 0;
  if (k.kind == COST_DENSE) {
    if (which == 0)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dense_rows<M_ROWSUM>, kThreads, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dense_cols, kThreads, 0);
  } else if (uses_direct_sweeps(k, prec)) {
    nb = direct_blocks_per_sm();
  } else {
    auto kern = which == 0 ? (k.zdot ? k_pts_sweep<M_ROWSUM, 0, false> : k_pts_sweep<M_ROWSUM, 0, true>)
                           : (k.zdot ? k_pts_sweep<M_COLSUM, 0, false> : k_pts_sweep<M_COLSUM, 0, true>);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, pts_smem(k.d));
  }
  return nb > 0 ? nb : 1;
}

// fixed / streamed points per CTA of each sweep (the split choice of lamp_create uses them)
int tile_outer(const Consts& k, int prec) {
  if (prec == 1 /* LAMP_PREC_BF16_TC */) return tc_tile_fixed();
  return k.kind == COST_DENSE ? kDR : uses_direct_sweeps(k, prec) ? direct_outer(k.d) : kPT;
}
int tile_inner(const Consts& k, int prec) {
  if (prec == 1) return tc_tile_stream();
  return k.kind == COST_DENSE ? kDChunk : uses_direct_sweeps(k, prec) ? kDirectTile : kPT;
}
int tile_outer_cols(const Consts& k, int prec) {
  if (prec == 1) return tc_tile_fixed();
  return k.kind == COST_DENSE ? kDChunk : uses_direct_sweeps(k, prec) ? direct_outer(k.d) : kPT;
}
int tile_inner_cols(const Consts& k, int prec) {
  if (prec == 1) return tc_tile_stream();
  return k.kind == COST_DENSE ? kDColRows : uses_direct_sweeps(k, prec) ? kDirectTile : kPT;
}

// gradient coordinates q0 .. q0 + DG - 1 (one recompute sweep per side)
template <int DG>
static cudaError_t launch_grad_d(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, float* dx,
                                 float* dy, int q0, cudaStream_t st) {
  if (dx) {
    // outer = rows (x), inner = columns (y): weights w_j of colq, outer offsets RqA of g2row
    SweepIO io;
    for (int b = 0; b < 2; ++b) { io.off2[b] = nullptr; io.off4[b] = w.g2row; io.indat[b] = w.colq[b]; }
    cudaError_t e = launch_pts<M_GRAD, DG>(in.x, in.y, k.n, k.m, k.d, io, w.rowpart, nullptr, g.rows_split, w.dev,
                                           k, st, nullptr, q0);
    if (e != cudaSuccess) return e;
    k_grad_fin<<<(unsigned)cdiv(k.n, 256), 256, 0, st>>>(w.rowpart, g.rows_split, k.n, DG, q0, k.d, in.x, in.r,
                                                        w.g2row, 1, k.s, dx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (dy) {
    // outer = columns (y), inner = rows (x): weights q_i of g2row, outer offsets BqA of colq
    SweepIO io;
    for (int b = 0; b < 2; ++b) { io.off2[b] = nullptr; io.off4[b] = w.colq[b]; io.indat[b] = w.g2row; }
    cudaError_t e = launch_pts<M_GRAD, DG>(in.y, in.x, k.m, k.n, k.d, io, w.colpart, nullptr, g.cols_split, w.dev,
                                           k, st, nullptr, q0);
    if (e != cudaSuccess) return e;
    k_grad_fin_cols<<<(unsigned)cdiv(k.m, 256), 256, 0, st>>>(w, g.cols_split, k.m, DG, q0, k.d, in.y, k.s, dy);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// the gradient in chunks of up to 8 coordinates (the partial-sum buffers hold 8 values per
// point when d > 8): ceil(d / 8) recompute sweeps per side
cudaError_t launch_grad(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec, float* dx,
                        float* dy, cudaStream_t st) {
  for (int q0 = 0; q0 < k.d; q0 += 8) {
    const int dg = k.d - q0 < 8 ? k.d - q0 : 8;
    cudaError_t e;
    switch (dg) {
      case 1: e = launch_grad_d<1>(in, k, w, g, dx, dy, q0, st); break;
      case 2: e = launch_grad_d<2>(in, k, w, g, dx, dy, q0, st); break;
      case 3: e = launch_grad_d<3>(in, k, w, g, dx, dy, q0, st); break;
      case 4: e = launch_grad_d<4>(in, k, w, g, dx, dy, q0, st); break;
      case 5: e = launch_grad_d<5>(in, k, w, g, dx, dy, q0, st); break;
      case 6: e = launch_grad_d<6>(in, k, w, g, dx, dy, q0, st); break;
      case 7: e = launch_grad_d<7>(in, k, w, g, dx, dy, q0, st); break;
      default: e = launch_grad_d<8>(in, k, w, g, dx, dy, q0, st); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------------------------------
// transport-map application (App. E, colour transfer): out = p V (side 0, V: m x k) or
// out = p^T U (side 1, U: n x k) for the current X^t = diag(r) p, 1 <= k <= 8

// out[i][q] = scale_i sum_s part[(s np + i) k + q], scale_i = src[i].y (/ div[i])
__global__ void k_map_fin(const double* __restrict__ part, int splits, int64_t np, int dk,
                          const float4* __restrict__ src, const double* __restrict__ div, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  double sc = (double)src[i].y;
  if (div) sc /= div[i];
  for (int q = 0; q < dk; ++q) {
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += part[((int64_t)s * np + i) * dk + q];
    out[i * dk + q] = (float)(sc * acc);
  }
}

// inner weights of side 1: 1 / S_i = q_i / r_i, in the g2row layout
__global__ void k_map_rowweights(const float4* __restrict__ g2row, const double* __restrict__ r, int64_t n,
                                 float4* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 g = g2row[i];
  out[i] = make_float4(g.x, (float)((double)g.y / r[i]), g.z, g.w);
}

// stored cost, side 0: one warp per row, sum_j 2^{v_ij} w_j V_j, times q_i / r_i
template <int DK>
__global__ void __launch_bounds__(kThreads)
k_dense_map_rows(const float* __restrict__ C, int64_t ldc, int64_t n, int64_t m, const float4* __restrict__ colq,
                 const float4* __restrict__ g2row, const double* __restrict__ r, const float* __restrict__ V,
                 float* __restrict__ out, const DevState* __restrict__ dev, const Consts k) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (i >= n) return;  // warp-uniform
  const SweepParams sp = make_sweep_params(sweep_kappa(dev->kappa, k), k);
  const float4 gr = g2row[i];
  const float* crow = C + i * ldc;
  double acc[DK];
#pragma unroll
  for (int q = 0; q < DK; ++q) acc[q] = 0.0;
  for (int64_t j0 = 0; j0 < m; j0 += 32 * 64) {
    float a[DK];
#pragma unroll
    for (int q = 0; q < DK; ++q) a[q] = 0.f;
    const int64_t j1 = j0 + 32 * 64 < m ? j0 + 32 * 64 : m;
    for (int64_t j = j0 + lane; j < j1; j += 32) {
      const float4 cd = colq[j];
      const float z = crow[j];
      const float v = __fmaf_rn(sp.alA, z, __fmaf_rn(sp.ahA, z, -(gr.x + cd.x)));
      const float e = ex2(v) * cd.y;
#pragma unroll
      for (int q = 0; q < DK; ++q) a[q] = __fmaf_rn(e, V[j * DK + q], a[q]);
    }
#pragma unroll
    for (int q = 0; q < DK; ++q) acc[q] += (double)a[q];
  }
  const double sc = (double)gr.y / r[i];
#pragma unroll
  for (int q = 0; q < DK; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) out[i * DK + q] = (float)(sc * v);
  }
}

// stored cost, side 1: one thread per column, sum_i 2^{v_ij} U_i / S_i, times w_j
template <int DK>
__global__ void __launch_bounds__(kThreads)
k_dense_map_cols(const float* __restrict__ C, int64_t ldc, int64_t n, int64_t m, const float4* __restrict__ colq,
                 const float4* __restrict__ g2row, const double* __restrict__ r, const float* __restrict__ U,
                 float* __restrict__ out, const DevState* __restrict__ dev, const Consts k) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const SweepParams sp = make_sweep_params(sweep_kappa(dev->kappa, k), k);
  const float4 cd = colq[j];
  double acc[DK];
#pragma unroll
  for (int q = 0; q < DK; ++q) acc[q] = 0.0;
  for (int64_t i0 = 0; i0 < n; i0 += 64) {
    float a[DK];
#pragma unroll
    for (int q = 0; q < DK; ++q) a[q] = 0.f;
    const int64_t i1 = i0 + 64 < n ? i0 + 64 : n;
    for (int64_t i = i0; i < i1; ++i) {
      const float4 gr = g2row[i];
      const float z = C[i * ldc + j];
      const float v = __fmaf_rn(sp.alA, z, __fmaf_rn(sp.ahA, z, -(gr.x + cd.x)));
      const float e = ex2(v) * (float)((double)gr.y / r[i]);
#pragma unroll
      for (int q = 0; q < DK; ++q) a[q] = __fmaf_rn(e, U[i * DK + q], a[q]);
    }
#pragma unroll
    for (int q = 0; q < DK; ++q) acc[q] += (double)a[q];
  }
#pragma unroll
  for (int q = 0; q < DK; ++q) out[j * DK + q] = (float)((double)cd.y * acc[q]);
}

template <int DK>
static cudaError_t launch_map_k(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int cur,
                                const float* V, float* out, int side, cudaStream_t st) {
  if (k.kind == COST_DENSE) {
    if (side == 0)
      k_dense_map_rows<DK><<<(unsigned)cdiv(k.n, kThreads / 32), kThreads, 0, st>>>(
          in.C, in.ldc, k.n, k.m, w.colq[cur], w.g2row, in.r, V, out, w.dev, k);
    else
      k_dense_map_cols<DK><<<(unsigned)cdiv(k.m, kThreads), kThreads, 0, st>>>(
          in.C, in.ldc, k.n, k.m, w.colq[cur], w.g2row, in.r, V, out, w.dev, k);
    return cudaGetLastError();
  }
  if (side == 0) {
    // outer = rows (x), inner = columns (y): weights w_j of colq, outer offsets RqA of g2row
    SweepIO io;
    for (int b = 0; b < 2; ++b) { io.off2[b] = nullptr; io.off4[b] = w.g2row; io.indat[b] = w.colq[b]; }
    cudaError_t e = launch_pts<M_GRAD, DK>(in.x, in.y, k.n, k.m, k.d, io, w.rowpart, nullptr, g.rows_split, w.dev,
                                           k, st, V);
    if (e != cudaSuccess) return e;
    k_map_fin<<<(unsigned)cdiv(k.n, 256), 256, 0, st>>>(w.rowpart, g.rows_split, k.n, DK, w.g2row, in.r, out);
    return cudaGetLastError();
  }
  // outer = columns (y), inner = rows (x) with weights 1 / S_i (in rowpart, free here)
  float4* rw = reinterpret_cast<float4*>(w.rowpart);
  k_map_rowweights<<<(unsigned)cdiv(k.n, 256), 256, 0, st>>>(w.g2row, in.r, k.n, rw);
  SweepIO io;
  for (int b = 0; b < 2; ++b) { io.off2[b] = nullptr; io.off4[b] = w.colq[b]; io.indat[b] = rw; }
  cudaError_t e = launch_pts<M_GRAD, DK>(in.y, in.x, k.m, k.n, k.d, io, w.colpart, nullptr, g.cols_split, w.dev, k,
                                         st, V);
  if (e != cudaSuccess) return e;
  k_map_fin<<<(unsigned)cdiv(k.m, 256), 256, 0, st>>>(w.colpart, g.cols_split, k.m, DK, w.colq[cur], nullptr, out);
  return cudaGetLastError();
}

cudaError_t launch_map(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int cur, const float* V,
                       int dk, float* out, int side, cudaStream_t st) {
  switch (dk) {
    case 1: return launch_map_k<1>(in, k, w, g, cur, V, out, side, st);
    case 2: return launch_map_k<2>(in, k, w, g, cur, V, out, side, st);
    case 3: return launch_map_k<3>(in, k, w, g, cur, V, out, side, st);
    case 4: return launch_map_k<4>(in, k, w, g, cur, V, out, side, st);
    case 5: return launch_map_k<5>(in, k, w, g, cur, V, out, side, st);
    case 6: return launch_map_k<6>(in, k, w, g, cur, V, out, side, st);
    case 7: return launch_map_k<7>(in, k, w, g, cur, V, out, side, st);
    case 8: return launch_map_k<8>(in, k, w, g, cur, V, out, side, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace lamp
