// Evaluation passes over the current X^t = diag(r) p^{eta_t}(nu^t) outside the
// iteration (arXiv 2511.11359):
//   * Round (Alg. 3, from Altschuler et al.) of X^t in factored form and the rounded
//     objective <C, Round(X^t)> of the certificate in Prop. infeas_bound (a);
//   * the dual function of the saddle problem (App. B): D(phi) for eta = 0 (row min)
//     and D^eta(phi) for eta > 0 (row softmin), Eqs. def:dual_spp and def:dual_spp_e.
// Both run the iteration's own sweeps on scratch column data: the state's other parity
// buffers (colq, colq2, rowshift of parity cur ^ 1), which the next iteration writes
// before it reads them.  Consts::same_kappa gives stream B stream A's exponents, so one
// sweep returns two weightings of the same entries; Consts::kap_ovr evaluates the
// sweeps at another kappa (the dual at kappa = 1/eta).
//
// Round of X = X^t.  row(X^t) = r by construction (Eq. row_feasible), so Step 1 has
// x_i = 1 and X' = X^t.  Step 2: y_j = min(c_j / A_j, 1) with A = col(X^t).  Step 3:
// delta_c_j = c_j - y_j A_j = max(c_j - A_j, 0), and delta_r_i = r_i - (X y)_i
// = r_i (sum_j X_ij (1 - y_j)) / r_i, which one row sweep gives as the ratio of two
// weightings of row i (weights w_j (1 - y_j) and w_j) without cancellation.  Step 4
// keeps the plan factored: Round(X^t) = X^t diag(y) + delta_r delta_c^T / ||delta_r||_1.
// Its cost: <C, X^t diag(y)> = sum_j y_j colz_j (+ sum_i s|x_i|^2 row''_i in the dot
// form), and delta_r^T C delta_c in closed form for |x - y|^2 (moments of delta_r and
// delta_c) or by one pass over a stored C.
#include <cmath>

#include "lamp_common.cuh"

namespace lamp {

namespace {

constexpr int kT = kFinThreads;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the block in a fixed order; the result is valid in thread 0
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r += sh[q];
  __syncthreads();
  return r;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// stream B's own row shift := stream A's (same exponent in both streams)
__global__ void k_same_shift(const float2* __restrict__ rs, float2* __restrict__ rs_s, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a = rs[i].x;
  rs_s[i] = make_float2(a, a);
}

// Round, Steps 2-3 on the columns.  Block partial fields (nf = 3 + dm):
//   0: sum y_j colz_j   1: sum delta_c_j   2: sum delta_c_j s|y_j|^2   3 + q: sum delta_c_j y_jq
__global__ void __launch_bounds__(kT)
k_round_cols(const Work w, int cur, const double* __restrict__ c, const float* __restrict__ ypts, int dm,
             float4* __restrict__ colq_s, float4* __restrict__ colq2_s, double* __restrict__ y_out,
             double* __restrict__ dc_out, double* __restrict__ dc_tmp, double* __restrict__ part, const Consts k) {
  __shared__ double sh[kT / 32];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double yc = 0.0, dc = 0.0, dcn = 0.0;
  if (j < k.m) {
    const double A = w.colA[j], cj = c[j];
    const bool over = A > cj;
    const double yj = over ? cj / A : 1.0;
    dc = over ? 0.0 : cj - A;
    const float4 cq = w.colq[cur][j];
    // weight of the second stream: w_j (1 - y_j) = w_j (A_j - c_j) / A_j
    const float wy = over ? (float)((double)cq.y * ((A - cj) / A)) : 0.0f;
    colq_s[j] = make_float4(cq.x, cq.y, cq.x, wy);
    // packed sweeps: stream B's term log2(w_j (1 - y_j)) (-inf where y_j = 1: no contribution)
    if (colq2_s) store_pair_entry(colq2_s, j, cq.x, cq.y, wy > 0.f ? (float)log2((double)wy) : -INFINITY, wy);
    yc = yj * w.colz[j];
    if (k.kind == COST_SQEUCLID) dcn = dc * k.s * w.ny[j];
    if (y_out) y_out[j] = yj;
    if (dc_out) dc_out[j] = dc;
    dc_tmp[j] = dc;
  }
  const int nf = 3 + dm;
  double r = block_sum(yc, sh);
  if (threadIdx.x == 0) part[blockIdx.x * nf + 0] = r;
  r = block_sum(dc, sh);
  if (threadIdx.x == 0) part[blockIdx.x * nf + 1] = r;
  r = block_sum(dcn, sh);
  if (threadIdx.x == 0) part[blockIdx.x * nf + 2] = r;
  for (int q = 0; q < dm; ++q) {
    r = block_sum(j < k.m ? dc * (double)ypts[j * dm + q] : 0.0, sh);
    if (threadIdx.x == 0) part[blockIdx.x * nf + 3 + q] = r;
  }
}

// Round, Step 3 on the rows, from the sweep with weights (w_j, w_j (1 - y_j)).  Fields:
//   0: sum delta_r_i   1: sum s|x_i|^2 row''_i (dot form)   2: sum delta_r_i s|x_i|^2
//   3 + q: sum delta_r_i x_iq
__global__ void __launch_bounds__(kT)
k_round_rows(const Work w, int splits, const double* __restrict__ r, const float* __restrict__ xpts, int dm,
             double* __restrict__ dr_out, double* __restrict__ part, const Consts k) {
  __shared__ double sh[kT / 32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double dr = 0.0, nrow = 0.0, drn = 0.0;
  if (i < k.n) {
    double S = 0.0, Sp = 0.0;
    for (int s = 0; s < splits; ++s) {
      S += w.rowpart[((int64_t)s * 2 + 0) * k.n + i];
      Sp += w.rowpart[((int64_t)s * 2 + 1) * k.n + i];
    }
    const double ri = r[i];
    dr = S > 0.0 ? ri * (Sp / S) : 0.0;
    if (k.kind == COST_SQEUCLID) {
      const double sn = k.s * w.nx[i];
      if (k.zdot) nrow = sn * (ri - dr);
      drn = dr * sn;
    }
    if (dr_out) dr_out[i] = dr;
    w.rowpart[i] = dr;  // kept for the stored-cost bilinear pass (only this thread reads index i)
  }
  const int nf = 3 + dm;
  double v = block_sum(dr, sh);
  if (threadIdx.x == 0) part[blockIdx.x * nf + 0] = v;
  v = block_sum(nrow, sh);
  if (threadIdx.x == 0) part[blockIdx.x * nf + 1] = v;
  v = block_sum(drn, sh);
  if (threadIdx.x == 0) part[blockIdx.x * nf + 2] = v;
  for (int q = 0; q < dm; ++q) {
    v = block_sum(i < k.n ? dr * (double)xpts[i * dm + q] : 0.0, sh);
    if (threadIdx.x == 0) part[blockIdx.x * nf + 3 + q] = v;
  }
}

// delta_r^T C delta_c for a stored cost: one warp per row, float32 products of the
// row of C with float32 delta_c, float64 accumulation per lane; per-row terms
// dr_i (C delta_c)_i go to rowterm[i]
__global__ void __launch_bounds__(kT)
k_round_dense_bilinear(const float* __restrict__ C, int64_t ldc, int64_t n, int64_t m,
                       const double* __restrict__ dr, const double* __restrict__ dc, double* __restrict__ rowterm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * (kT / 32) + wid;
  if (i >= n) return;  // warp-uniform
  const float* row = C + i * ldc;
  double acc = 0.0;
  for (int64_t j0 = 0; j0 < m; j0 += 32 * 32) {
    float a = 0.f;
    const int64_t j1 = j0 + 32 * 32 < m ? j0 + 32 * 32 : m;
    for (int64_t j = j0 + lane; j < j1; j += 32) a = __fmaf_rn(row[j], (float)dc[j], a);
    acc += (double)a;
  }
  acc = warp_sum(acc);
  if (lane == 0) rowterm[i] = acc * dr[i];
}

// delta_r^T C delta_c for a point-cloud cost without a closed form (l1, l-inf): one warp
// per row, the cost recomputed in float32, float64 accumulation per lane
__global__ void __launch_bounds__(kT)
k_round_pts_bilinear(const float* __restrict__ x, const float* __restrict__ y, int d, int64_t n, int64_t m,
                     const double* __restrict__ dr, const double* __restrict__ dc, double* __restrict__ rowterm,
                     const Consts k) {
  __shared__ float sx[kT / 32][64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * (kT / 32) + wid;
  if (i >= n) return;  // warp-uniform; no block-wide barrier below
  for (int q = lane; q < d; q += 32) sx[wid][q] = x[i * d + q];
  __syncwarp();
  double acc = 0.0;
  for (int64_t j0 = 0; j0 < m; j0 += 32 * 32) {
    float a = 0.f;
    const int64_t j1 = j0 + 32 * 32 < m ? j0 + 32 * 32 : m;
    for (int64_t j = j0 + lane; j < j1; j += 32) {
      float z = 0.f;
      for (int q = 0; q < d; ++q) {
        const float ad = fabsf(sx[wid][q] - y[j * d + q]);
        z = k.cost_op == 1 ? z + ad : fmaxf(z, ad);
      }
      a = __fmaf_rn(z, (float)dc[j], a);
    }
    acc += (double)a;
  }
  acc = warp_sum(acc);
  if (lane == 0) rowterm[i] = k.s * acc * dr[i];
}

// out[q] = sum over blocks b of part[b * nf + q], in a fixed order (one block per field)
__global__ void __launch_bounds__(kT) k_fields(const double* __restrict__ part, int64_t nblocks, int nf,
                                               double* __restrict__ out) {
  __shared__ double sh[kT / 32];
  const int q = blockIdx.x;
  double v = 0.0;
  for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x) v += part[b * nf + q];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) out[q] = v;
}

__global__ void k_round_final(const double* __restrict__ rowf, const double* __restrict__ colf,
                              const double* __restrict__ densef, int dm, const Consts k, double* __restrict__ out) {
  const double ndr = rowf[0], ndc = colf[1];
  const double cpp = colf[0] + rowf[1];  // <C, X^t diag(y)>
  double bil;
  if (k.kind == COST_SQEUCLID && k.cost_op == 0) {
    // sum_ij s |x_i - y_j|^2 dr_i dc_j = (sum dr s|x|^2)(sum dc) + (sum dr)(sum dc s|y|^2) - 2 s (sum dr x).(sum dc y)
    double cross = 0.0;
    for (int q = 0; q < dm; ++q) cross += rowf[3 + q] * colf[3 + q];
    bil = rowf[2] * ndc + ndr * colf[2] - 2.0 * k.s * cross;
  } else {
    bil = densef[0];  // stored cost, or l1 / l-inf point costs: one pass
  }
  out[0] = cpp + (ndr > 0.0 ? bil / ndr : 0.0);
  out[1] = ndr;
  out[2] = ndc;
  out[3] = cpp;
}

// dual bound: column data of phi (theta^t or nu^t) at the sweep parameters of k (same
// kappa in both streams); field 0: sum_j c_j phi_j
__global__ void __launch_bounds__(kT)
k_dual_cols(const Work w, int cur, int which, const double* __restrict__ c, float4* __restrict__ colq_s,
            float4* __restrict__ colq2_s, double* __restrict__ part, const Consts k) {
  __shared__ double sh[kT / 32];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (j < k.m) {
    const double phi = which ? w.nu[cur][j] : w.theta[cur][j];
    const SweepParams sp = make_sweep_params(k.kap_ovr, k);
    const double sny = k.zdot ? k.s * w.ny[j] : 0.0;
    if (k.eta > 0.0) {
      float dB;
      const float4 cd = column_data(phi, phi, sny, sp, k, &dB);
      colq_s[j] = cd;
      if (colq2_s) store_pair_entry(colq2_s, j, cd.x, cd.y, dB, cd.w);
    } else {
      // eta = 0: the row-max passes read {Bq_j, Br_j} (the offset on the grid and the
      // remainder Br_j = Bcol_j - Bq_j, |Br_j| <= g/2, as a float) instead of a weight
      const double b = sp.lamA * (sny + 2.0 * k.K * phi);
      const double q = quantize(b, sp.g);
      colq_s[j] = make_float4((float)q, (float)(b - q), (float)q, (float)(b - q));
      // the same in the packed-pair layout, which the tensor-core row-max passes read
      if (colq2_s) store_pair_entry(colq2_s, j, (float)q, (float)(b - q), 0.f, (float)(b - q));
    }
    v = c[j] * phi;
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// dual bound, rows: eta = 0 from the row maxima of the prime pass, eta > 0 from the
// row sums; field 0: sum_i r_i rowmin_i
__global__ void __launch_bounds__(kT)
k_dual_rows(const Work w, const float2* __restrict__ rs_s, int splits, const double* __restrict__ r, int soft,
            double* __restrict__ part, const Consts k) {
  __shared__ double sh[kT / 32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < k.n) {
    const SweepParams sp = make_sweep_params(k.kap_ovr, k);
    const double snx = k.zdot ? k.s * w.nx[i] : 0.0;
    double mn;
    if (!soft) {
      // refinement pass: M = max_j (a z_ij - Bq_j - Br_j - Rq_i)
      //                    = -lambda (min_j (C_ij + 2K phi_j) - s|x_i|^2 [dot form]) - Rq_i
      float M = -INFINITY;
      for (int s = 0; s < splits; ++s) M = fmaxf(M, w.rowmax[((int64_t)s * 2 + 0) * k.n + i]);
      mn = -((double)rs_s[i].x + (double)M) / sp.lamA + snx;
    } else {
      // softmin = -(1/kappa) log Z_i, log2 Z_i = Rq_i - lambda s|x_i|^2 + log2 S_i
      double S = 0.0;
      for (int s = 0; s < splits; ++s) S += w.rowpart[((int64_t)s * 2 + 0) * k.n + i];
      const double L2 = (double)rs_s[i].x - sp.lamA * snx + log2(S);
      mn = -kLn2 * L2 / sp.kapA;
    }
    v = r[i] * mn;
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

}  // namespace

cudaError_t launch_round(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec, int cur,
                         double* out4, double* y, double* dr, double* dc, cudaStream_t st) {
  const int nx = cur ^ 1;  // scratch parity
  // the closed-form bilinear term needs the coordinate moments (|x - y|^2 only)
  const bool moments = k.kind == COST_SQEUCLID && k.cost_op == 0;
  const int dm = moments ? k.d : 0;
  const int nf = 3 + dm;
  const int64_t rb = fin_blocks(k.n), cb = fin_blocks(k.m);
  double* rowp = w.rscr;
  double* colp = rowp + rb * nf;
  double* rowf = colp + cb * nf;
  double* colf = rowf + nf;
  double* densef = colf + nf;
  // delta_c for the stored-cost bilinear pass: colpart is free during an evaluation
  double* dc_tmp = w.colpart;

  k_same_shift<<<(unsigned)cdiv(k.n, kT), kT, 0, st>>>(w.rowshift[cur], w.rowshift[nx], k.n);
  k_round_cols<<<(unsigned)cb, kT, 0, st>>>(w, cur, in.c, in.y, dm, w.colq[nx], w.colq2[nx], y, dc, dc_tmp, colp,
                                           k);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // row sweep over X^t with column weights (w_j, w_j (1 - y_j)), both at kappa_t
  Consts k2 = k;
  k2.same_kappa = 1;
  Work w2 = w;
  w2.colq[0] = w2.colq[1] = w.colq[nx];
  w2.colq2[0] = w2.colq2[1] = w.colq2[nx];
  w2.rowshift[0] = w2.rowshift[1] = w.rowshift[nx];
  e = launch_iteration_part(in, k2, w2, g, prec, 0, 0, st);
  if (e != cudaSuccess) return e;
  k_round_rows<<<(unsigned)rb, kT, 0, st>>>(w, g.rows_split, in.r, in.x, dm, dr, rowp, k);
  if (!moments) {
    // delta_r is in rowpart[0, n) (k_round_rows); per-row terms go to rowpart[n, 2n)
    if (k.kind == COST_DENSE)
      k_round_dense_bilinear<<<(unsigned)cdiv(k.n, kT / 32), kT, 0, st>>>(in.C, in.ldc, k.n, k.m, w.rowpart,
                                                                         dc_tmp, w.rowpart + k.n);
    else
      k_round_pts_bilinear<<<(unsigned)cdiv(k.n, kT / 32), kT, 0, st>>>(in.x, in.y, k.d, k.n, k.m, w.rowpart,
                                                                        dc_tmp, w.rowpart + k.n, k);
    k_fields<<<1, kT, 0, st>>>(w.rowpart + k.n, k.n, 1, densef);
  }
  k_fields<<<(unsigned)nf, kT, 0, st>>>(rowp, rb, nf, rowf);
  k_fields<<<(unsigned)nf, kT, 0, st>>>(colp, cb, nf, colf);
  k_round_final<<<1, 1, 0, st>>>(rowf, colf, densef, dm, k, out4);
  return cudaGetLastError();
}

cudaError_t launch_dual(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec, int cur,
                        int which, double* out2, cudaStream_t st) {
  const int nx = cur ^ 1;
  const int64_t rb = fin_blocks(k.n), cb = fin_blocks(k.m);
  double* rowp = w.rscr;
  double* colp = rowp + rb;
  double* res = colp + cb;
  Consts k2 = k;
  k2.same_kappa = 1;
  // eta > 0: the softmin at kappa = 1/eta; eta = 0: the row min, from two row-max passes
  // at a large kappa (the second with the row shifts of the first and the column
  // remainders subtracted)
  const bool soft = k.eta > 0.0;
  k2.kap_ovr = soft ? 1.0 / k.eta : 65536.0 / k.K;
  Work w2 = w;
  w2.colq[0] = w2.colq[1] = w.colq[nx];
  w2.colq2[0] = w2.colq2[1] = w.colq2[nx];
  w2.rowshift[0] = w2.rowshift[1] = w.rowshift[nx];
  k_dual_cols<<<(unsigned)cb, kT, 0, st>>>(w, cur, which, in.c, w.colq[nx], w.colq2[nx], colp, k2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_prime(in, k2, w2, g, prec, st);
  if (e != cudaSuccess) return e;
  if (soft) {
    e = launch_iteration_part(in, k2, w2, g, prec, 0, 0, st);
    if (e != cudaSuccess) return e;
  } else {
    // second pass with the primed row shifts: near each row's maximum |u| is a few grid
    // steps, so its float32 rounding (and that of the remainder) is ~2^-24 g, and the row
    // minimum min_j (C_ij + 2K phi_j) of the kernels' cost comes out with an absolute error
    // of order 2^-46 W instead of W 2^-24 (W the offset bound, a few K)
    e = launch_rowmax_refined(in, k2, w2, g, prec, st);
    if (e != cudaSuccess) return e;
  }
  k_dual_rows<<<(unsigned)rb, kT, 0, st>>>(w, w.rowshift[nx], g.rows_split, in.r, soft ? 1 : 0, rowp, k2);
  k_fields<<<1, kT, 0, st>>>(rowp, rb, 1, res);
  k_fields<<<1, kT, 0, st>>>(colp, cb, 1, res + 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(out2, res, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

}  // namespace lamp
