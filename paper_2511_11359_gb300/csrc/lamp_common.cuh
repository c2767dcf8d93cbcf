// Shared definitions of the LAMP CUDA library (device side + host launch glue).
//
// Notation (arXiv 2511.11359):
//   K = ||C||_inf, kappa_t = 1/eta_t (kappa_0 = 0), s = cost scale.
//   Stream A of iteration t is (kappa_t, nu^t)            -> X^t       (Alg. 2, thetabar step)
//   Stream B of iteration t is (kappa_{t+1}, nubar^{t+1}) -> Xbar^{t+1} (Alg. 2, thetahat step)
//   Both only depend on (nu^t, theta^t, kappa_t), so one pass over the (i,j)
//   pairs serves both streams.
//
// Compensated base-2 exponent.  With lambda = kappa * log2(e), the exponent of
// p^{eta}(nu)_ij is, in base 2 and up to the row normaliser,
//     s2_ij = -lambda (C_ij + 2K nu_j).
// The kernels evaluate it as v_ij = a z_ij - Bq_j - Rq_i where
//   direct form (DENSE, and SQEUCLID with d <= 8):
//             z = C_ij / s (stored cost, or sum_k (x_ik - y_jk)^2),
//             a = -lambda s,  Bcol_j = lambda 2K nu_j,  Rrow_i = M_i
//   dot form (SQEUCLID with d > 8):
//             z = x_i . y_j,  a = 2 lambda s,  Bcol_j = lambda (s|y_j|^2 + 2K nu_j),
//                                              Rrow_i = lambda s |x_i|^2 + M_i
// The direct form's float32 error is relative to C_ij itself; the dot form's is
// relative to |x_i||y_j|, which is what tensor cores (and d = 64) need.
// with M_i a per-row shift (a running estimate of log2 of the row maximum).
// Bq_j and Rq_i are Bcol_j, Rrow_i rounded to a power-of-two grid g chosen so
// that |Bq| + |Rq| < 2^23 g: their float32 sum is then exact, the product a z
// is exact inside the FMA, and a = ah + al (two floats) keeps kappa's float64
// precision.  v therefore carries one float32 rounding relative to |v| itself
// (|v| = O(1) for the entries that matter), instead of relative to
// lambda |C| = O(t), which is what a naive float32 exponent would give at
// eta = 0 where kappa_t = t/(2K) grows without bound (Section 3.2).
// The sub-grid remainder Br_j = Bcol_j - Bq_j enters as the factor
// w_j = 2^{-Br_j} (row sums) or as a per-column factor after the sum (column sums).
//
// Shared row shift (packed sweeps, Consts::shared_shift): stream B uses stream A's
// row shift, RqB_i = RqA_i, and its exponent is derived from stream A's as
// v^B = (a^B - a^A) z + (v^A + dB_j) with dB_j = BqA_j - BcolB_j (BcolB unquantised,
// so the column weight of stream B is inside the exponent).  dB_j is O(1):
// kappa_{t+1} nubar_j and kappa_t nu_j differ by O(tau1), so v^B - v^A = O(1) for
// every entry, the row sums of stream B stay within a few powers of two of 1, and
// the rounding of v^A + dB_j is relative to O(1) numbers.  The row sweep then sums
// 2^{v^B} with no weight, and the column finalize takes stream B's column sum as is.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lamp {

constexpr double kLog2e = 1.4426950408889634074;
constexpr double kLn2 = 0.69314718055994530942;

enum CostKind : int { COST_DENSE = 0, COST_SQEUCLID = 1 };

// threads per block of the O(n + m) finalize kernels; rowred / colred hold one partial
// per block.  Their time is the float64 instruction latency of one thread's chain (the
// FP64 rate of this part is ~1/64 of FP32), so smaller blocks do not make them faster.
constexpr int kFinThreads = 128;
inline int64_t fin_blocks(int64_t len) { return (len + kFinThreads - 1) / kFinThreads; }
// doubles of Work::rscr: per-block partials of up to 4 + d fields for rows and columns,
// the reduced fields and the results
inline size_t rscr_doubles(int64_t n, int64_t m, int d) {
  return (size_t)(fin_blocks(n) + fin_blocks(m) + 2) * (size_t)(4 + d) + 256;
}

// Problem constants, fixed for the lifetime of a context (passed by value).
struct Consts {
  int64_t n, m;
  int32_t d, kind;
  double K;          // ||C||_inf of the cost in use
  double s;          // cost scale (1 for DENSE)
  double tau1, tau2, eta, alpha;
  double clipb;      // tanh(beta/2)
  double alpha_m;    // alpha / m (c^alpha = c + alpha/m, Section 3.1)
  double W;          // bound factor for the exponent offsets: |Bq|+|Rq| <= lambda*W + 128
  double rnx;        // sum_i r_i s |x_i|^2 (dot-form cost bookkeeping), 0 otherwise
  int32_t zdot;      // 1: z = x.y (dot form), 0: z = C/s (direct form)
  int32_t shared_shift;  // 1: both streams use stream A's row shift (packed direct-form sweeps)
  // evaluation passes outside the iteration (rounding, dual bound) run the sweeps on
  // scratch column data with these set: kap_ovr >= 0 replaces kappa_t, and
  // same_kappa = 1 gives stream B stream A's kappa (two weightings of one exponent)
  double kap_ovr = -1.0;
  int32_t same_kappa = 0;
  // point-cloud ground cost of the direct form: 0 |x - y|^2, 1 sum_k |x_k - y_k| (l1),
  // 2 max_k |x_k - y_k| (l-inf)
  int32_t cost_op = 0;
  // eta > 0: 1 = the termination rule uses the infeasibility alone (no kappa condition)
  int32_t infeas_only = 0;
};

// Parameters of one iteration's sweeps, derived from kappa_t alone.
struct SweepParams {
  double kapA, kapB;   // kappa_t, kappa_{t+1}
  double lamA, lamB;   // kappa * log2(e)
  double aA, aB;       // float64 exponent multipliers of z
  float ahA, alA, ahB, alB;  // a = ah + al, both float32
  double g;            // offset grid (power of two)
  double wB;           // tau1 / kappa_{t+1} = tau1 eta_{t+1}, the averaging weight of Alg. 2
};

__host__ __device__ inline double kappa_next(double kap, const Consts& k) {
  // 1/eta_{t+1} = tau1 + (1/eta_t)(1 - tau1 eta)   (Alg. 2, Section 3.2)
  return k.tau1 + kap * (1.0 - k.tau1 * k.eta);
}

// kappa of the sweeps: the state's, unless an evaluation pass overrides it
__host__ __device__ inline double sweep_kappa(double dev_kappa, const Consts& k) {
  return k.kap_ovr >= 0.0 ? k.kap_ovr : dev_kappa;
}

__host__ __device__ inline SweepParams make_sweep_params(double kap, const Consts& k) {
  SweepParams p;
  p.kapA = kap;
  p.kapB = k.same_kappa ? kap : kappa_next(kap, k);
  p.lamA = p.kapA * kLog2e;
  p.lamB = p.kapB * kLog2e;
  if (!k.zdot) {
    p.aA = -p.lamA * k.s;
    p.aB = -p.lamB * k.s;
  } else {
    p.aA = 2.0 * p.lamA * k.s;
    p.aB = 2.0 * p.lamB * k.s;
  }
  p.wB = k.tau1 / p.kapB;
  p.ahA = (float)p.aA;
  p.alA = (float)(p.aA - (double)p.ahA);
  p.ahB = (float)p.aB;
  p.alB = (float)(p.aB - (double)p.ahB);
  double lmax = p.lamA > p.lamB ? p.lamA : p.lamB;
  double bound = lmax * k.W + 128.0;
  // smallest e with 2^e >= bound (bound = f 2^ex, f in [0.5, 1)), then g = 2^(e-23)
  int ex;
  const double f = frexp(bound, &ex);
  const int e = f == 0.5 ? ex - 1 : ex;
  p.g = ldexp(1.0, e - 23);
  return p;
}

// round-to-nearest multiple of the power-of-two grid g, exact in float64
__host__ __device__ inline double quantize(double x, double g) {
  // g is a power of two, so x * (1 / g) == x / g exactly (and avoids a float64 division)
  const double ginv = 1.0 / g;
#ifdef __CUDA_ARCH__
  return rint(x * ginv) * g;
#else
  return __builtin_rint(x * ginv) * g;
#endif
}

#ifdef __CUDACC__
// write entry e of a packed-pair array (layout described in Work)
__device__ __forceinline__ void store_pair_entry(float4* __restrict__ a, int64_t e, float offA, float wA, float dB,
                                                 float wB) {
  float* fa = reinterpret_cast<float*>(a + (e >> 1) * 2);
  const int h = (int)(e & 1);
  fa[0 + h] = -offA;
  fa[2 + h] = wA;
  fa[4 + h] = dB;
  fa[6 + h] = wB;
}

// stream B's term of entry e of a column pair array: dB_e = BqA_e - BcolB_e
__device__ __forceinline__ float pair_dB(const float4* __restrict__ a, int64_t e) {
  return reinterpret_cast<const float*>(a + (e >> 1) * 2 + 1)[e & 1];
}

// 2^x with the SFU (MUFU.EX2), flush-to-zero
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// packed pairs of floats (fma / add / sub / mul .rn.f32x2: two IEEE round-to-nearest
// operations per instruction, lane by lane identical to the scalar ones)
__device__ __forceinline__ uint64_t pk(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk(uint64_t v) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(v));
  return f;
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// 2^v for a pair of entries: v = al z + (ah z + o), o = -(Rq + Bq) exact (see the top of this file)
__device__ __forceinline__ uint64_t exp2_pair(uint64_t ah2, uint64_t al2, uint64_t z2, uint64_t o2) {
  const float2 v = upk(f2fma(al2, z2, f2fma(ah2, z2, o2)));
  return pk(ex2(v.x), ex2(v.y));
}

// the column data {BqA, wA, BqB, wB} of one column for sweep parameters sp: Bcol of
// each stream rounded to the grid, and the factor 2^{-remainder}; *dB (if given) gets
// BqA - BcolB, stream B's term under the shared row shift (see the top of this file)
__device__ __forceinline__ float4 column_data(double nu_j, double nubar_j, double sny_j, const SweepParams& sp,
                                              const Consts& k, float* dB = nullptr) {
  double bA = sp.lamA * (sny_j + 2.0 * k.K * nu_j);
  double bB = sp.lamB * (sny_j + 2.0 * k.K * nubar_j);
  double qA = quantize(bA, sp.g);
  double qB = quantize(bB, sp.g);
  if (dB) *dB = (float)(qA - bB);
  // the sub-grid remainders are at most half a grid step: their powers of two in float32
  return make_float4((float)qA, exp2f((float)(qA - bA)), (float)qB, exp2f((float)(qB - bB)));
}

// Visit the per-split partials of one point in split order: ld(s) loads split s's values,
// use(v) consumes them.  The loads are issued in groups of 8 before any of them is used: a
// loop over a run-time number of splits below its unroll factor would otherwise issue one
// load per trip, each behind the add of the previous one.
template <typename LD, typename USE>
__device__ __forceinline__ void for_splits(int splits, LD&& ld, USE&& use) {
  using V = decltype(ld(0));
  for (int s0 = 0; s0 < splits; s0 += 8) {
    V v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (s0 + u < splits) v[u] = ld(s0 + u);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (s0 + u < splits) use(v[u]);
  }
}

// Knuth's branch-free TwoSum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// accumulate x into the float-float pair (hi, lo)
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  hi = s;
  lo += e;
}

// warp sum of float-float values (hi, lo): TwoSum of the high parts, low parts and their
// errors added; the sweeps' per-thread sums are reduced in float32 arithmetic (the FP64
// rate of this part is a small fraction of FP32) and converted once
__device__ __forceinline__ void warp_sum_ff(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float sum, err;
    two_sum(hi, h2, sum, err);
    hi = sum;
    lo = lo + l2 + err;
  }
}
#endif

// Device-resident control block of one context.
// float32 constants the sweeps take from make_sweep_params (a = ah + al per stream, and
// a^B - a^A for the shared row shift)
struct SweepF {
  float ahA, alA, ahB, alB, dal;
  float pad[3];
};

struct DevState {
  long long t;        // iteration index of the current state
  double kappa;       // kappa_t
  int cur;            // which of the two state buffers holds state t
  int done;           // set: the remaining launches of a device loop return at once
  int status;         // 0 or LAMP_E_NUMERIC
  int eval_only;      // 1: compute the pass but never apply the update
  double tol;         // stop at the first t >= 1 with res <= tol (and, for eta > 0, 1 - kappa eta <= tol)
  long long tmax;     // stop when t >= tmax
  unsigned int ticket;  // last-block counter of the column finalize kernel
  unsigned int pad;
  // results for the last evaluated X^t
  long long t_eval;
  double kappa_eval;
  double res;         // ||col(X^t) - c||_1 (+ ||row(X^t) - r||_1 = 0 by construction)
  double costA;       // <C, X^t>
  double colnu;       // <col(X^t), nu^t>
  double rlogZ;       // <r, log Z^t>
  // the iteration's parameters at kappa = swf_kap (make_sweep_params of kappa_t and of
  // kappa_{t+1}, and the sweeps' float32 constants), written once per iteration by the
  // column finalize; swf_kap = -1 (never equal to kappa >= 0) until then
  double swf_kap;
  SweepF swf;
  SweepParams spc, spn;
};

__host__ __device__ inline SweepF sweep_floats(const SweepParams& p) {
  SweepF f;
  f.ahA = p.ahA;
  f.alA = p.alA;
  f.ahB = p.ahB;
  f.alB = p.alB;
  f.dal = (float)(p.aB - p.aA);
  f.pad[0] = f.pad[1] = f.pad[2] = 0.f;
  return f;
}

#ifdef __CUDACC__
// the sweeps' constants at the current kappa: from the control block when the column
// finalize of the previous iteration computed them for this kappa, else (first iteration
// after a state change, evaluation passes with a kappa override) derived here in float64
__device__ __forceinline__ SweepF sweep_floats_of(const DevState* dev, const Consts& k) {
  if (k.kap_ovr < 0.0 && !k.same_kappa) {
    const double kap = dev->kappa;
    if (dev->swf_kap == kap) return dev->swf;
    return sweep_floats(make_sweep_params(kap, k));
  }
  return sweep_floats(make_sweep_params(sweep_kappa(dev->kappa, k), k));
}

// make_sweep_params of kappa_t and kappa_{t+1} for the finalize kernels (cached as above)
__device__ __forceinline__ void iteration_params_of(const DevState* dev, const Consts& k, SweepParams& sp,
                                                    SweepParams& spn) {
  const double kap = dev->kappa;
  if (k.kap_ovr < 0.0 && !k.same_kappa && dev->swf_kap == kap) {
    sp = dev->spc;
    spn = dev->spn;
  } else {
    sp = make_sweep_params(kap, k);
    spn = make_sweep_params(sp.kapB, k);
  }
}
#endif

// Device buffers of one context (all owned by the context).
struct Work {
  double* nu[2];
  double* theta[2];
  float4* colq[2];     // per column {BqA, wA, BqB, wB}
  float2* rowshift[2]; // per row {RqA, RqB}
  float4* g2row;       // per row {RqA, qA, RqB, qB} for the column sweep
  // the same data in the packed-pair layout read by the packed sweeps (null when unused):
  // for entries 2p, 2p+1 two float4, [2p] = {-offA_2p, -offA_2p+1, wgtA_2p, wgtA_2p+1}
  // and [2p+1] = {dB_2p, dB_2p+1, wgtB_2p, wgtB_2p+1}: columns dB = BqA - BcolB, the
  // term stream B adds to stream A's exponent under the shared row shift; rows dB = 0
  // (unused); padding halves hold {-2^100, 0}
  float4* colq2[2];
  float4* g2row2;
  double* rowpart;     // [splits_rows][2][n] partial row sums
  double* colpart;     // [splits_cols][3][m] partial column sums (A, B, cost-weighted A)
  double* logZ;        // [n] natural-log normalisers of X^t
  double* colA;        // [m] col(X^t)
  double* colz;        // [m] sum_i C_ij X_ij of the last pass that accumulated the cost, without
                       // the dot form's sum_i s|x_i|^2 X_ij (added by its users)
  double* rscr;        // reduction scratch of the rounding / dual-bound passes
  double* nx;          // [n] |x_i|^2 (SQEUCLID)
  double* ny;          // [m] |y_j|^2 (SQEUCLID)
  double* rowred;      // [rowfin blocks] partial <r, log Z>
  double* colred;      // [colfin blocks][3] partial (res, cost, colnu)
  float* rowmax;       // [splits_rows][2][n] partial row maxima (prime pass)
  double* scratch;     // small reduction scratch (K pass, marginal checks)
  DevState* dev;
};

// Launch geometry chosen at create time.
struct Geometry {
  const void* map_x;  // tensor maps of the bf16 point copies (LAMP_PREC_BF16_TC), else null:
  const void* map_y;  // 128-row boxes (fixed tiles) ...
  const void* map_x64;  // ... and 64-row boxes (streamed tiles)
  const void* map_y64;
  const void* map_c;  // tensor map of a stored cost for the TMA-fed sweeps (LAMP_COST_DENSE), else null
  int sms;
  int rows_split;   // inner splits of the row sweep
  int cols_split;   // inner splits of the column sweep
  int rows_tiles;   // outer tiles of the row sweep
  int cols_tiles;   // outer tiles of the column sweep
};

struct Inputs {
  const float* C;
  int64_t ldc;
  const float* x;
  const float* y;
  const double* r;
  const double* c;
};

// ---- launchers (lamp_kernels.cu) ----
cudaError_t launch_norms(const Inputs& in, const Consts& k, const Work& w, cudaStream_t st);
// cosine cost: out_i = P_i / (sqrt 2 |P_i|); rows with a zero or non-finite norm are counted in *bad
cudaError_t launch_unit_rows(const float* P, int64_t np, int d, float* out, unsigned int* bad, cudaStream_t st);
cudaError_t launch_kmax(const Inputs& in, const Consts& k, const Work& w, const Geometry& g,
                        int prec, cudaStream_t st);
cudaError_t launch_check_marginals(const Inputs& in, const Consts& k, const Work& w, cudaStream_t st);
cudaError_t launch_init_state(const Inputs& in, const Consts& k, const Work& w, int zero, cudaStream_t st);
cudaError_t launch_prime(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                         cudaStream_t st);
// after launch_prime: per row and split, max_j (v_ij - Br_j) with the primed row shifts
// applied (Work::rowmax, stream A slot); the column data's second field holds Br_j
cudaError_t launch_rowmax_refined(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                                  cudaStream_t st);
// eval = 1: an evaluation pass, whose column sweep also accumulates <C, X^t> (the
// packed direct-form column sweep leaves it out of the regular iterations)
cudaError_t launch_iteration(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                             int eval, cudaStream_t st);
void prepare_kernels();
// tcgen05 path (lamp_tc.cu)
size_t tc_smem_bytes();
int64_t tc_pad(int64_t v);
cudaError_t tc_convert(const float* P, int64_t np, int d, float* Pr, void* Pb, cudaStream_t st);
cudaError_t tc_fill_pads(float4* a, int64_t from, int64_t to, cudaStream_t st);
cudaError_t tc_fill_pairs(float4* a, int64_t count, cudaStream_t st);
cudaError_t tc_make_map(void* map_out, const void* base, int64_t rows_pad, int box_rows);
// stored-cost sweeps fed by TMA (lamp_dense.cu)
cudaError_t dense_make_map(void* map_out, const float* C, int64_t n, int64_t m, int64_t ldc);
cudaError_t dense_prepare();
int dense_tile_rows();
int dense_tile_cols();
int dense_blocks_per_sm();
cudaError_t dense_launch_sweep(bool rows, int eval, const Geometry& g, const Work& w, const Consts& k, int splits,
                               cudaStream_t st);
// tensor-core gradient pass (lamp_tc_grad.cu): transposed bf16 copies (64 x np_pad), one side
// of the pass (float32 partials [splits][np][64]) and its finalize
size_t tcg_smem_bytes();
cudaError_t tcg_prepare();
cudaError_t tcg_transpose(const void* Pb, int64_t np_pad, void* PT, cudaStream_t st);
int tcg_tile_fixed();
int tcg_tile_stream();
cudaError_t tcg_launch(bool rows, const void* map_fixed, const void* map_stream, const void* map_streamT,
                       const Work& w, const Consts& k, int splits, float* part, cudaStream_t st);
cudaError_t tcg_finalize(bool rows, const float* part, int splits, const Work& w, const Consts& k, const float* P,
                         const double* r, const float4* wsrc, float* out, cudaStream_t st);
// 2-D bf16 tensor map over a row-major (rows x inner) array with box_inner x box_rows boxes
// and 128-byte swizzle (inner * 2 bytes a multiple of 16)
cudaError_t tc_make_map2(void* map_out, const void* base, int64_t inner, int64_t rows, int box_inner, int box_rows);
int tc_tile_fixed();   // points of the fixed tile of a tensor-core sweep
int tc_tile_stream();  // points of a streamed tile
cudaError_t tc_prepare();
// self-test of the bounded mbarrier wait (0, or a LAMP_E_* code); *status = the device status word
int tc_wait_selftest(uint32_t polls, int* status);
int tc_blocks_per_sm(int which);
// eval = 1: the column sweep of an evaluation pass (with the cost-weighted sums)
cudaError_t tc_launch_sweep(bool rows, int eval, const Geometry& g, const Work& w, const Consts& k, int splits,
                            cudaStream_t st);
cudaError_t tc_launch_rowmax(int mode, const Geometry& g, const Work& w, const Consts& k, int splits, cudaStream_t st);
cudaError_t launch_iteration_part(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                                  int part, int eval, cudaStream_t st);
int tile_outer_cols(const Consts& k, int prec);
int tile_inner_cols(const Consts& k, int prec);
cudaError_t launch_grad(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec,
                        float* dx, float* dy, cudaStream_t st);
// transport-map application (lamp_kernels.cu): out = p V (side 0) or p^T U (side 1), 1 <= dk <= 8
cudaError_t launch_map(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int cur, const float* V,
                       int dk, float* out, int side, cudaStream_t st);
// evaluation passes (lamp_eval.cu); `cur` is the state-buffer parity, read by the host beforehand.
// Round: out4 (device, 4 doubles) = {<C, Round(X^t)>, ||delta_r||_1, ||delta_c||_1, <C, X''>}
cudaError_t launch_round(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec, int cur,
                         double* out4, double* y, double* dr, double* dc, cudaStream_t st);
// dual bound at theta^t (which = 0) or nu^t (which = 1): out2 (device) = {sum_i r_i rowmin_i,
// <c, phi>}, with rowmin the row min (eta = 0) or row softmin (eta > 0) of C_ij + 2K phi_j
cudaError_t launch_dual(const Inputs& in, const Consts& k, const Work& w, const Geometry& g, int prec, int cur,
                        int which, double* out2, cudaStream_t st);
int launches_per_iteration(const Consts& k, int prec);
// record a message for lamp_last_error(NULL) (errors raised without a context)
void set_last_error_null(const char* msg);
int sweep_blocks_per_sm(const Consts& k, int prec, int which);
int tile_outer(const Consts& k, int prec);
int tile_inner(const Consts& k, int prec);
// whether the packed direct-form sweeps serve this problem (then Consts::shared_shift = 1)
bool uses_direct_sweeps(const Consts& k, int prec);
// packed direct-form sweeps (lamp_direct.cu): inner tile, outer points per CTA, occupancy, launch
constexpr int kDirectTile = 128;
int direct_outer(int d);
int direct_blocks_per_sm();
cudaError_t launch_direct_sweep(bool rows, int eval, const Inputs& in, const Consts& k, const Work& w,
                                const Geometry& g, cudaStream_t st);

}  // namespace lamp
