// Host side of the LAMP C ABI (include/lamp.h): validation, the O(n + m) workspace,
// the device loop (CUDA graphs of whole iterations, polled every check_every
// iterations) and the O(1) bookkeeping of the objective (App. D identity,
// Prop. infeas_bound (a)).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lamp.h"
#include "lamp_common.cuh"

using namespace lamp;

struct lamp_ctx {
  Consts k{};
  Work w{};
  Geometry g{};
  Inputs in{};
  int prec = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream used for graph capture
  lamp_params params{};
  double Hr = 0.0;             // entropy of r
  double log_m = 0.0;
  int rowblocks = 0;
  int part_width = 3;  // values per point the partial-sum buffers hold (per split)
  std::vector<void*> allocs;
  // owned input copies (lamp_create_owned)
  bool owned = false;
  float* own_a = nullptr;  // C or x
  float* own_b = nullptr;  // y
  double* own_r = nullptr;
  double* own_c = nullptr;
  // graph slots: 0 = one iteration, 1 = check_every iterations, 2 = one evaluation pass
  cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};
  int64_t glen[3] = {0, 0, 0};
  DevState* host_dev = nullptr;  // pinned mirror for polling
  // LAMP_PREC_BF16_TC: bf16 copies (zero padded to 128-row multiples x 64 coordinates),
  // float32 copies of the rounded points, and their TMA descriptors
  void* xb = nullptr;
  void* yb = nullptr;
  // the public cost kind; LAMP_COST_COSINE: unit-scaled copies of the points (see lamp.h)
  int pub_kind = 0;
  float* xn = nullptr;
  float* yn = nullptr;
  float* xr = nullptr;
  float* yr = nullptr;
  alignas(64) unsigned char map_x[128];
  alignas(64) unsigned char map_y[128];
  alignas(64) unsigned char map_x64[128];
  alignas(64) unsigned char map_y64[128];
  alignas(64) unsigned char map_c[128];  // stored cost (TMA-fed sweeps)
  // tensor-core gradient pass (LAMP_PREC_BF16_TC, |x - y|^2): transposed bf16 copies of the
  // points (64 x n_pad, 64 x m_pad), their tensor maps and the float32 partial sums
  void* xT = nullptr;
  void* yT = nullptr;
  bool tcg_fresh = false;  // the transposed copies match the current bf16 points
  float* tcg_part = nullptr;
  size_t tcg_part_floats = 0;
  cudaStream_t gside = nullptr;  // the gradient's second side runs on this stream
  cudaEvent_t gfork = nullptr, gjoin = nullptr;
  alignas(64) unsigned char map_xT[128];
  alignas(64) unsigned char map_yT[128];
  std::string err;
};

static thread_local std::string g_err;

void lamp::set_last_error_null(const char* msg) { g_err = msg ? msg : ""; }

static int fail(lamp_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_err = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess)                                                                \
      return fail(ctx, _e == cudaErrorMemoryAllocation ? LAMP_E_NOMEM : LAMP_E_CUDA,      \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, __LINE__);  \
  } while (0)

template <class T>
static int dalloc(lamp_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return fail(ctx, LAMP_E_NOMEM, "cudaMalloc(%zu bytes): %s", count * sizeof(T),
                                    cudaGetErrorString(e));
  ctx->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return LAMP_OK;
}

extern "C" int lamp_params_default(lamp_params* p) {
  if (!p) return fail(nullptr, LAMP_E_INVALID, "lamp_params_default: null pointer");
  std::memset(p, 0, sizeof(*p));
  p->eta = 0.0;
  p->tau1 = 0.0;
  p->tau2 = 0.0;
  p->alpha = 0.01;
  p->beta = 1.1;
  p->tol = 1e-6;
  p->max_iter = 100000;
  p->check_every = 50;
  p->prec = LAMP_PREC_FP32;
  p->infeas_only = 0;
  p->K = 0.0;
  p->gap_tol = 0.0;
  p->gap_every = 0;
  return LAMP_OK;
}

// host-side validation that needs no device (so that it is testable without a GPU)
static int validate(const lamp_problem* pr, const lamp_params* pa, bool device_ptrs) {
  if (!pr || !pa) return fail(nullptr, LAMP_E_INVALID, "null problem or params");
  if (pr->n < 1 || pr->m < 1) return fail(nullptr, LAMP_E_INVALID, "n and m must be >= 1 (n=%lld m=%lld)",
                                         (long long)pr->n, (long long)pr->m);
  if (pr->n > (int64_t(1) << 31) || pr->m > (int64_t(1) << 31))
    return fail(nullptr, LAMP_E_INVALID, "n and m must be <= 2^31");
  if ((double)pr->n * (double)pr->m >= 4.0e18) return fail(nullptr, LAMP_E_INVALID, "n*m too large");
  if (pr->kind < LAMP_COST_DENSE || pr->kind > LAMP_COST_COSINE)
    return fail(nullptr, LAMP_E_INVALID, "unknown cost kind %d", pr->kind);
  if (!pr->r || !pr->c) return fail(nullptr, LAMP_E_INVALID, "r and c must be non-null");
  if (pr->kind == LAMP_COST_DENSE) {
    if (!pr->C) return fail(nullptr, LAMP_E_INVALID, "DENSE cost needs C");
    if (pr->ldc < pr->m) return fail(nullptr, LAMP_E_INVALID, "ldc (%lld) < m (%lld)", (long long)pr->ldc,
                                     (long long)pr->m);
  } else {
    if (!pr->x || !pr->y) return fail(nullptr, LAMP_E_INVALID, "point-cloud costs need x and y");
    if (pr->d < 1 || pr->d > 64) return fail(nullptr, LAMP_E_INVALID, "d must be in [1, 64] (d=%lld)",
                                             (long long)pr->d);
    if (!std::isfinite(pr->cost_scale)) return fail(nullptr, LAMP_E_INVALID, "cost_scale must be finite");
  }
  if (!(pa->eta >= 0.0) || !std::isfinite(pa->eta)) return fail(nullptr, LAMP_E_INVALID, "eta must be >= 0");
  if (!(pa->tau1 >= 0.0) || !(pa->tau2 >= 0.0) || !std::isfinite(pa->tau1) || !std::isfinite(pa->tau2))
    return fail(nullptr, LAMP_E_INVALID, "tau1, tau2 must be >= 0 (0 = 1/(2K))");
  if (!(pa->alpha > 0.0) || !std::isfinite(pa->alpha)) return fail(nullptr, LAMP_E_INVALID, "alpha must be > 0");
  if (!(pa->beta > 0.0) || !std::isfinite(pa->beta)) return fail(nullptr, LAMP_E_INVALID, "beta must be > 0");
  if (std::isnan(pa->tol)) return fail(nullptr, LAMP_E_INVALID, "tol is NaN");
  if (pa->max_iter < 0) return fail(nullptr, LAMP_E_INVALID, "max_iter must be >= 0");
  if (pa->check_every < 1 || pa->check_every > 100000)
    return fail(nullptr, LAMP_E_INVALID, "check_every must be in [1, 100000]");
  if (pa->prec != LAMP_PREC_FP32 && pa->prec != LAMP_PREC_BF16_TC)
    return fail(nullptr, LAMP_E_INVALID, "unknown precision %d", pa->prec);
  if (pa->prec == LAMP_PREC_BF16_TC && pr->kind != LAMP_COST_SQEUCLID && pr->kind != LAMP_COST_COSINE)
    return fail(nullptr, LAMP_E_INVALID, "LAMP_PREC_BF16_TC applies to LAMP_COST_SQEUCLID and LAMP_COST_COSINE only");
  if (!(pa->K >= 0.0) || !std::isfinite(pa->K)) return fail(nullptr, LAMP_E_INVALID, "K must be >= 0");
  if (pa->tau1 > 0.0 && pa->tau1 * pa->eta > 1.0) return fail(nullptr, LAMP_E_INVALID, "tau1 * eta must be <= 1");
  if (!(pa->gap_tol >= 0.0) || !std::isfinite(pa->gap_tol))
    return fail(nullptr, LAMP_E_INVALID, "gap_tol must be >= 0 and finite (0 = no gap test)");
  if (pa->gap_every < 0) return fail(nullptr, LAMP_E_INVALID, "gap_every must be >= 0 (0 = check_every)");
  if (pa->infeas_only != 0 && pa->infeas_only != 1) return fail(nullptr, LAMP_E_INVALID, "infeas_only must be 0 or 1");
  (void)device_ptrs;
  return LAMP_OK;
}

static int choose_split(int64_t tout, int64_t tin, int64_t wave, int64_t min_inner, double per_split = 0.002) {
  int best = 1;
  double best_score = -1.0;
  int64_t smax = std::min<int64_t>(std::max<int64_t>(tin / std::max<int64_t>(min_inner, 1), 1), 128);
  for (int s = 1; s <= smax; ++s) {
    int64_t ctas = tout * s;
    int64_t waves = (ctas + wave - 1) / wave;
    double util = (double)ctas / (double)(waves * wave);
    double score = util - per_split * s;
    if (score > best_score + 1e-12) {
      best_score = score;
      best = s;
    }
  }
  return best;
}

static int build_graph(lamp_ctx* ctx, int slot, int64_t len) {
  if (ctx->gexec[slot] && ctx->glen[slot] == len) return LAMP_OK;
  if (ctx->gexec[slot]) {
    cudaGraphExecDestroy(ctx->gexec[slot]);
    ctx->gexec[slot] = nullptr;
  }
  CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
  for (int64_t i = 0; i < len; ++i) {
    cudaError_t e = launch_iteration(ctx->in, ctx->k, ctx->w, ctx->g, ctx->prec, slot == 2, ctx->cap);
    if (e != cudaSuccess) {
      cudaGraph_t gg;
      cudaStreamEndCapture(ctx->cap, &gg);
      if (gg) cudaGraphDestroy(gg);
      return fail(ctx, LAMP_E_CUDA, "capturing an iteration: %s", cudaGetErrorString(e));
    }
  }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamEndCapture(ctx->cap, &graph));
  cudaError_t e = cudaGraphInstantiate(&ctx->gexec[slot], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(ctx, LAMP_E_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  ctx->glen[slot] = len;
  return LAMP_OK;
}

__global__ void k_ctrl(DevState* dev, int eval_only, double tol, long long tmax_abs, long long tmax_rel, int set) {
  dev->done = 0;
  dev->eval_only = eval_only;
  dev->tol = tol;
  dev->tmax = tmax_rel >= 0 ? dev->t + tmax_rel : tmax_abs;
  dev->ticket = 0u;
  if (set) dev->status = 0;
}

__global__ void k_mark_done(DevState* dev) { dev->done = 1; }

__global__ void k_set_state(DevState* dev, long long t, double kappa) {
  dev->t = t;
  dev->kappa = kappa;
  dev->swf_kap = -1.0;  // the sweeps derive their constants until the next column finalize
  dev->done = 0;
  dev->status = 0;
  dev->ticket = 0u;
  dev->t_eval = -1;
}

static int poll(lamp_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->host_dev, ctx->w.dev, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LAMP_OK;
}

static int prime(lamp_ctx* ctx) {
  // column data of the current buffer, then row shifts from a coarse row-max pass
  CK(launch_init_state(ctx->in, ctx->k, ctx->w, 0, ctx->stream));
  CK(launch_prime(ctx->in, ctx->k, ctx->w, ctx->g, ctx->prec, ctx->stream));
  return LAMP_OK;
}

static int create_impl(lamp_ctx** out, const lamp_problem* prob, const lamp_params* params, void* stream,
                       bool owned) {
  if (!out) return fail(nullptr, LAMP_E_INVALID, "lamp_create: out is null");
  *out = nullptr;
  int rc = validate(prob, params, !owned);
  if (rc) return rc;
  lamp_ctx* ctx = new lamp_ctx();
  ctx->params = *params;
  ctx->prec = params->prec;
  ctx->stream = (cudaStream_t)stream;
  auto bail = [&](int code) {
    lamp_destroy(ctx);
    return code;
  };
  {
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) {
      fail(nullptr, LAMP_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
      delete ctx;
      return LAMP_E_CUDA;
    }
  }
  prepare_kernels();
  if (params->prec == LAMP_PREC_BF16_TC) {
    cudaError_t e = tc_prepare();
    if (e != cudaSuccess) {
      fail(nullptr, LAMP_E_CUDA, "tcgen05 kernel setup: %s", cudaGetErrorString(e));
      delete ctx;
      return LAMP_E_CUDA;
    }
  }
  Consts& k = ctx->k;
  // point-cloud kinds run as COST_SQEUCLID internally with a ground-cost op (l1, l-inf) or
  // on unit-scaled points (cosine)
  const bool pts = prob->kind != LAMP_COST_DENSE;
  ctx->pub_kind = prob->kind;
  k.n = prob->n;
  k.m = prob->m;
  k.d = pts ? (int32_t)prob->d : 0;
  k.kind = pts ? COST_SQEUCLID : COST_DENSE;
  k.cost_op = prob->kind == LAMP_COST_L1 ? 1 : prob->kind == LAMP_COST_LINF ? 2 : 0;
  // direct-form cost (z = |x - y|^2) for small d; dot form x.y above (|x - y|^2 only)
  k.zdot = (pts && k.cost_op == 0 && (prob->d > 8 || params->prec == LAMP_PREC_BF16_TC)) ? 1 : 0;
  // the packed sweeps (direct form and tensor cores) derive stream B from stream A
  k.shared_shift = (uses_direct_sweeps(k, params->prec) || params->prec == LAMP_PREC_BF16_TC) ? 1 : 0;
  k.eta = params->eta;
  k.infeas_only = params->infeas_only;
  k.alpha = params->alpha;
  k.alpha_m = params->alpha / (double)prob->m;
  k.clipb = std::tanh(params->beta / 2.0);
  ctx->log_m = std::log((double)k.m);

  if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess) {
    fail(nullptr, LAMP_E_CUDA, "cudaStreamCreate failed");
    delete ctx;
    return LAMP_E_CUDA;
  }
  // inputs
  Inputs& in = ctx->in;
  if (owned) {
    ctx->owned = true;
    size_t na = prob->kind == LAMP_COST_DENSE ? (size_t)prob->n * prob->m : (size_t)prob->n * prob->d;
    if ((rc = dalloc(ctx, &ctx->own_a, na))) return bail(rc);
    if (pts && (rc = dalloc(ctx, &ctx->own_b, (size_t)prob->m * prob->d)))
      return bail(rc);
    if ((rc = dalloc(ctx, &ctx->own_r, (size_t)prob->n))) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->own_c, (size_t)prob->m))) return bail(rc);
    cudaError_t e = cudaSuccess;
    if (prob->kind == LAMP_COST_DENSE) {
      e = cudaMemcpy2DAsync(ctx->own_a, prob->m * sizeof(float), prob->C, prob->ldc * sizeof(float),
                            prob->m * sizeof(float), prob->n, cudaMemcpyHostToDevice, ctx->stream);
    } else {
      e = cudaMemcpyAsync(ctx->own_a, prob->x, na * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->own_b, prob->y, (size_t)prob->m * prob->d * sizeof(float), cudaMemcpyHostToDevice,
                            ctx->stream);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->own_r, prob->r, prob->n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->own_c, prob->c, prob->m * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "input copy: %s", cudaGetErrorString(e)));
    in.C = prob->kind == LAMP_COST_DENSE ? ctx->own_a : nullptr;
    in.ldc = prob->m;
    in.x = pts ? ctx->own_a : nullptr;
    in.y = ctx->own_b;
    in.r = ctx->own_r;
    in.c = ctx->own_c;
  } else {
    in.C = prob->C;
    in.ldc = prob->ldc;
    in.x = prob->x;
    in.y = prob->y;
    in.r = prob->r;
    in.c = prob->c;
  }

  // geometry
  Geometry& g = ctx->g;
  {
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, ctx->device);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e)));
    g.sms = prop.multiProcessorCount;
  }
  {
    const bool tcp = ctx->prec == LAMP_PREC_BF16_TC;
    int bpr = tcp ? tc_blocks_per_sm(0) : sweep_blocks_per_sm(k, ctx->prec, 0);
    int bpc = tcp ? tc_blocks_per_sm(1) : sweep_blocks_per_sm(k, ctx->prec, 1);
    int64_t to = (k.n + tile_outer(k, ctx->prec) - 1) / tile_outer(k, ctx->prec);
    int64_t ti = (k.m + tile_inner(k, ctx->prec) - 1) / tile_inner(k, ctx->prec);
    int64_t tco = (k.m + tile_outer_cols(k, ctx->prec) - 1) / tile_outer_cols(k, ctx->prec);
    int64_t tci = (k.n + tile_inner_cols(k, ctx->prec) - 1) / tile_inner_cols(k, ctx->prec);
    g.rows_tiles = (int)to;
    g.cols_tiles = (int)tco;
    // at least 4 inner tiles per CTA (dense rows: 2 chunks of 1024 columns), so that a
    // CTA's fixed costs (parameters, reduction) stay small against its sweep; a problem
    // whose grid would not fill a quarter of one wave takes one tile per CTA instead
    // (n = m = 256 points: 2 CTAs instead of 1 per sweep)
    int min_inner = k.kind == LAMP_COST_DENSE ? 2 : 4;
    const auto mi = [&](int64_t tout, int64_t tin, int64_t wave, int base) {
      return tout * std::max<int64_t>(tin / base, 1) * 4 < wave ? 1 : base;
    };
    // a split costs 0.2 % of a wave in the score (0.06 % for the tensor-core sweeps, whose
    // CTAs carry little fixed cost: at n = m = 2^15 19 splits, exactly 8 waves of 304 CTAs,
    // beat 7 splits, 2.95 waves, by 1.4 % per iteration including the finalizes' longer sums)
    const double per_split = tcp ? 0.0006 : 0.002;
    g.rows_split = choose_split(to, ti, (int64_t)g.sms * bpr, mi(to, ti, (int64_t)g.sms * bpr, min_inner), per_split);
    g.cols_split = choose_split(tco, tci, (int64_t)g.sms * bpc,
                                mi(tco, tci, (int64_t)g.sms * bpc, k.kind == LAMP_COST_DENSE ? 4 : min_inner),
                                per_split);
    if (k.kind == LAMP_COST_DENSE && dense_make_map(ctx->map_c, in.C, k.n, k.m, in.ldc) == cudaSuccess &&
        dense_prepare() == cudaSuccess) {
      // a stored cost with a 16-byte aligned base and rows a multiple of 16 bytes apart:
      // the TMA-fed sweeps (32 x 256 tiles), at least 8 tiles per CTA for the copy ring
      g.map_c = ctx->map_c;
      const int64_t tr = dense_tile_rows(), tcl = dense_tile_cols();
      const int64_t wave = (int64_t)g.sms * dense_blocks_per_sm();
      g.rows_split = choose_split((k.n + tr - 1) / tr, (k.m + tcl - 1) / tcl, wave, 8);
      g.cols_split = choose_split((k.m + tcl - 1) / tcl, (k.n + tr - 1) / tr, wave, 8);
    }
  }

  // workspace
  Work& w = ctx->w;
  const size_t n = (size_t)k.n, m = (size_t)k.m;
  ctx->rowblocks = (int)fin_blocks(k.n);
  int colblocks = (int)fin_blocks(k.m);
  // partial-sum width: the sweeps' 2 / 3 values per point, and the gradient's d values;
  // the transport map widens the buffers on first use (ensure_part_width)
  const size_t gradd = k.kind == COST_SQEUCLID ? (size_t)std::min<int64_t>(std::max<int64_t>(k.d, 2), 8) : 2;
  ctx->part_width = (int)std::max<size_t>(3, gradd);
  // the bf16 point copies are padded to whole 128-point units (tc_pad); the per-point
  // column / row data to whole tiles of every sweep (a multiple of 256: the stored-cost
  // row sweep reads the data of 256 columns per tile); padding entries contribute nothing
  const size_t m_pad = (size_t)tc_pad(k.m), n_pad = (size_t)tc_pad(k.n);
  const size_t pm_pad = (m_pad + 255) / 256 * 256, pn_pad = (n_pad + 255) / 256 * 256;
  for (int b = 0; b < 2; ++b) {
    if ((rc = dalloc(ctx, &w.nu[b], m))) return bail(rc);
    if ((rc = dalloc(ctx, &w.theta[b], m))) return bail(rc);
    if ((rc = dalloc(ctx, &w.colq[b], pm_pad))) return bail(rc);
    if ((rc = dalloc(ctx, &w.rowshift[b], n))) return bail(rc);
  }
  if ((rc = dalloc(ctx, &w.g2row, pn_pad))) return bail(rc);
  if (ctx->prec == LAMP_PREC_BF16_TC || k.shared_shift) {
    for (int b = 0; b < 2; ++b)
      if ((rc = dalloc(ctx, &w.colq2[b], pm_pad))) return bail(rc);
    if ((rc = dalloc(ctx, &w.g2row2, pn_pad))) return bail(rc);
  }
  if ((rc = dalloc(ctx, &w.rowpart, (size_t)g.rows_split * ctx->part_width * n))) return bail(rc);
  if ((rc = dalloc(ctx, &w.colpart, (size_t)g.cols_split * ctx->part_width * m))) return bail(rc);
  if ((rc = dalloc(ctx, &w.logZ, n))) return bail(rc);
  if ((rc = dalloc(ctx, &w.colA, m))) return bail(rc);
  if ((rc = dalloc(ctx, &w.colz, m))) return bail(rc);
  if ((rc = dalloc(ctx, &w.rscr, rscr_doubles(k.n, k.m, k.kind == LAMP_COST_SQEUCLID ? (int)k.d : 0)))) return bail(rc);
  if ((rc = dalloc(ctx, &w.nx, n))) return bail(rc);
  if ((rc = dalloc(ctx, &w.ny, m))) return bail(rc);
  if ((rc = dalloc(ctx, &w.rowred, (size_t)ctx->rowblocks))) return bail(rc);
  if ((rc = dalloc(ctx, &w.colred, (size_t)colblocks * 3))) return bail(rc);
  if ((rc = dalloc(ctx, &w.rowmax, (size_t)g.rows_split * 2 * n))) return bail(rc);
  if ((rc = dalloc(ctx, &w.scratch, (size_t)std::max(3 * 4 * g.sms, 3 * 128)))) return bail(rc);
  if ((rc = dalloc(ctx, &w.dev, 1))) return bail(rc);
  {
    cudaError_t e = cudaMallocHost(&ctx->host_dev, sizeof(DevState));
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_NOMEM, "cudaMallocHost: %s", cudaGetErrorString(e)));
  }
  std::memset(ctx->host_dev, 0, sizeof(DevState));
  ctx->host_dev->swf_kap = -1.0;  // no cached sweep constants yet (kappa >= 0 always)
  ctx->host_dev->t_eval = -1;
  {
    cudaError_t e = cudaMemcpyAsync(w.dev, ctx->host_dev, sizeof(DevState), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "init copy: %s", cudaGetErrorString(e)));
    tc_fill_pads(w.colq[0], k.m, (int64_t)pm_pad, ctx->stream);
    tc_fill_pads(w.colq[1], k.m, (int64_t)pm_pad, ctx->stream);
    tc_fill_pads(w.g2row, k.n, (int64_t)pn_pad, ctx->stream);
    if (w.g2row2) {
      tc_fill_pairs(w.colq2[0], (int64_t)pm_pad, ctx->stream);
      tc_fill_pairs(w.colq2[1], (int64_t)pm_pad, ctx->stream);
      tc_fill_pairs(w.g2row2, (int64_t)pn_pad, ctx->stream);
    }
    cudaMemsetAsync(w.nu[0], 0, m * sizeof(double), ctx->stream);
    cudaMemsetAsync(w.theta[0], 0, m * sizeof(double), ctx->stream);
    cudaMemsetAsync(w.nu[1], 0, m * sizeof(double), ctx->stream);
    cudaMemsetAsync(w.theta[1], 0, m * sizeof(double), ctx->stream);
  }

  // marginals: positive, finite, summing to one (r in Delta^n, c in Delta^m, full support)
  {
    cudaError_t e = launch_check_marginals(in, k, w, ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "marginal check: %s", cudaGetErrorString(e)));
    std::vector<double> h(3 * 128);
    e = cudaMemcpyAsync(h.data(), w.scratch, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "marginal check: %s", cudaGetErrorString(e)));
    for (int which = 0; which < 2; ++which) {
      double S = 0, M = INFINITY, B = 0;
      for (int b = 0; b < 64; ++b) {
        S += h[which * 192 + 3 * b];
        M = std::min(M, h[which * 192 + 3 * b + 1]);
        B = std::max(B, h[which * 192 + 3 * b + 2]);
      }
      if (B != 0.0 || !(M > 0.0) || std::fabs(S - 1.0) > 1e-9)
        return bail(fail(ctx, LAMP_E_INVALID, "%s must be positive, finite and sum to 1 (sum-1=%.3e, min=%.3e)",
                         which ? "c" : "r", S - 1.0, M));
    }
  }
  // H(r) on the host needs r: copy it once (O(n))
  {
    std::vector<double> hr(n);
    cudaError_t e = cudaMemcpyAsync(hr.data(), in.r, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "copy r: %s", cudaGetErrorString(e)));
    double H = 0.0;
    for (double v : hr) H -= v * std::log(v);
    ctx->Hr = H;
  }

  // cosine cost: every kernel reads unit-scaled copies u = x / (sqrt 2 |x|), v = y / (sqrt 2 |y|)
  // (then |u - v|^2 = 1 - cos(x, y), see lamp.h)
  if (ctx->pub_kind == LAMP_COST_COSINE) {
    if ((rc = dalloc(ctx, &ctx->xn, n * (size_t)k.d))) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->yn, m * (size_t)k.d))) return bail(rc);
    unsigned int* bad = reinterpret_cast<unsigned int*>(w.scratch);
    unsigned int hbad = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), ctx->stream);
    if (e == cudaSuccess) e = launch_unit_rows(in.x, k.n, k.d, ctx->xn, bad, ctx->stream);
    if (e == cudaSuccess) e = launch_unit_rows(in.y, k.m, k.d, ctx->yn, bad, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "cosine normalisation: %s", cudaGetErrorString(e)));
    if (hbad) return bail(fail(ctx, LAMP_E_INVALID, "cosine cost needs nonzero finite points (%u are not)", hbad));
    in.x = ctx->xn;
    in.y = ctx->yn;
  }

  // bf16 copies for the tensor-core sweeps; the float32 kernels (K pass, prime pass,
  // gradient) then read the float32 copies of the rounded points, so every kernel
  // solves the problem of the rounded points
  if (ctx->prec == LAMP_PREC_BF16_TC) {
    if ((rc = dalloc(ctx, reinterpret_cast<uint16_t**>(&ctx->xb), n_pad * 64))) return bail(rc);
    if ((rc = dalloc(ctx, reinterpret_cast<uint16_t**>(&ctx->yb), m_pad * 64))) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->xr, n * (size_t)k.d))) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->yr, m * (size_t)k.d))) return bail(rc);
    cudaError_t e = tc_convert(in.x, k.n, k.d, ctx->xr, ctx->xb, ctx->stream);
    if (e == cudaSuccess) e = tc_convert(in.y, k.m, k.d, ctx->yr, ctx->yb, ctx->stream);
    if (e == cudaSuccess) e = tc_make_map(ctx->map_x, ctx->xb, (int64_t)n_pad, tc_tile_fixed() / 2);
    if (e == cudaSuccess) e = tc_make_map(ctx->map_y, ctx->yb, (int64_t)m_pad, tc_tile_fixed() / 2);
    if (e == cudaSuccess) e = tc_make_map(ctx->map_x64, ctx->xb, (int64_t)n_pad, tc_tile_stream());
    if (e == cudaSuccess) e = tc_make_map(ctx->map_y64, ctx->yb, (int64_t)m_pad, tc_tile_stream());
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "bf16 setup: %s", cudaGetErrorString(e)));
    in.x = ctx->xr;
    in.y = ctx->yr;
    g.map_x = ctx->map_x;
    g.map_y = ctx->map_y;
    g.map_x64 = ctx->map_x64;
    g.map_y64 = ctx->map_y64;
  }

  // cost scale and K = ||C||_inf of the cost the kernels use
  {
    cudaError_t e = launch_norms(in, k, w, ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "norms: %s", cudaGetErrorString(e)));
    bool need_K = !(params->K > 0.0);
    bool need_scale = pts && prob->cost_scale < 0.0;
    double s = pts ? (prob->cost_scale > 0.0 ? prob->cost_scale : 1.0) : 1.0;
    double Dmax = NAN, Dmin = NAN;
    if (need_K || need_scale || prob->kind == LAMP_COST_DENSE) {
      k.K = 1.0;
      k.s = s;
      e = launch_kmax(in, k, w, g, ctx->prec, ctx->stream);
      if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "K pass: %s", cudaGetErrorString(e)));
      if (prob->kind == LAMP_COST_DENSE) {
        std::vector<double> h(3 * 4 * g.sms);
        e = cudaMemcpyAsync(h.data(), w.scratch, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "K pass: %s", cudaGetErrorString(e)));
        Dmax = -INFINITY;
        Dmin = INFINITY;
        double bad = 0;
        for (int b = 0; b < 4 * g.sms; ++b) {
          Dmax = std::max(Dmax, h[3 * b]);
          Dmin = std::min(Dmin, h[3 * b + 1]);
          bad = std::max(bad, h[3 * b + 2]);
        }
        if (bad != 0.0 || !(Dmin >= 0.0))
          return bail(fail(ctx, LAMP_E_INVALID, "C must be finite and >= 0 (min %.3e)", Dmin));
      } else {
        std::vector<float> h((size_t)g.rows_split * 2 * n);
        e = cudaMemcpyAsync(h.data(), w.rowmax, h.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "K pass: %s", cudaGetErrorString(e)));
        float mx = -INFINITY, mnneg = -INFINITY;
        for (int sp = 0; sp < g.rows_split; ++sp)
          for (size_t i = 0; i < n; ++i) {
            mx = std::max(mx, h[(sp * 2 + 0) * n + i]);
            mnneg = std::max(mnneg, h[(sp * 2 + 1) * n + i]);
          }
        Dmax = mx;
        Dmin = -(double)mnneg;
        if (!std::isfinite(Dmax)) return bail(fail(ctx, LAMP_E_INVALID, "points must be finite"));
      }
    }
    if (need_scale) {
      if (!(Dmax > 0.0)) return bail(fail(ctx, LAMP_E_INVALID, "cost_scale < 0 needs a positive maximum cost"));
      s = 1.0 / Dmax;
    }
    k.s = s;
    double Kc = prob->kind == LAMP_COST_DENSE ? Dmax : s * std::max(Dmax, -Dmin);
    k.K = need_K ? Kc : params->K;
    if (!(k.K > 0.0) || !std::isfinite(k.K))
      return bail(fail(ctx, LAMP_E_INVALID, "||C||_inf must be positive and finite (got %g)", k.K));
  }
  k.tau1 = params->tau1 > 0.0 ? params->tau1 : 1.0 / (2.0 * k.K);
  k.tau2 = params->tau2 > 0.0 ? params->tau2 : 1.0 / (2.0 * k.K);
  if (k.tau1 * k.eta > 1.0) return bail(fail(ctx, LAMP_E_INVALID, "tau1 * eta must be <= 1"));

  // offset bound factor W: |Bq_j| + |Rq_i| <= lambda W + 128 (see lamp_common.cuh)
  if (!k.zdot) {
    k.W = 5.0 * k.K;
    k.rnx = 0.0;
  } else {
    std::vector<double> hx(n), hy(m), hr(n);
    cudaError_t e = cudaMemcpyAsync(hx.data(), w.nx, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hy.data(), w.ny, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hr.data(), in.r, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "norm copy: %s", cudaGetErrorString(e)));
    double nxm = 0, nym = 0, rnx = 0;
    for (size_t i = 0; i < n; ++i) {
      nxm = std::max(nxm, hx[i]);
      rnx += hr[i] * hx[i];
    }
    for (size_t j = 0; j < m; ++j) nym = std::max(nym, hy[j]);
    k.W = k.s * (nxm + 3.0 * nym) + 4.0 * k.K + 2.0 * k.s * (nxm + nym);
    k.rnx = k.s * rnx;
  }

  if ((rc = prime(ctx))) return bail(rc);
  {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, LAMP_E_CUDA, "create: %s", cudaGetErrorString(e)));
  }
  *out = ctx;
  return LAMP_OK;
}

extern "C" int lamp_create(lamp_ctx** out, const lamp_problem* prob, const lamp_params* params, void* stream) {
  return create_impl(out, prob, params, stream, false);
}

extern "C" int lamp_create_owned(lamp_ctx** out, const lamp_problem* prob, const lamp_params* params,
                                 void* stream) {
  return create_impl(out, prob, params, stream, true);
}

static int run_graph(lamp_ctx* ctx, int slot, int64_t len) {
  int rc = build_graph(ctx, slot, len);
  if (rc) return rc;
  CK(cudaGraphLaunch(ctx->gexec[slot], ctx->stream));
  return LAMP_OK;
}

static void fill_result(lamp_ctx* ctx, lamp_result* out, int stop, double gap) {
  if (!out) return;
  const DevState& d = *ctx->host_dev;
  out->iters = d.t;
  out->infeas = d.res;
  out->obj_CX = d.costA;
  out->kappa = d.kappa;
  out->K = ctx->k.K;
  out->status = d.status;
  out->stop = stop;
  out->gap = gap;
}

static int evaluate(lamp_ctx* ctx);
static int objective_values(lamp_ctx* ctx, double* out);

extern "C" int lamp_solve(lamp_ctx* ctx, lamp_result* out) {
  if (!ctx) return fail(nullptr, LAMP_E_INVALID, "lamp_solve: null context");
  const lamp_params& pa = ctx->params;
  auto arm = [&]() {
    k_ctrl<<<1, 1, 0, ctx->stream>>>(ctx->w.dev, 0, pa.tol, pa.max_iter, -1, 0);
    return cudaGetLastError();
  };
  CK(arm());
  const int64_t L = pa.check_every;
  // primal-dual gap test (App. E.2): every gap_every iterations (a multiple of the polling
  // interval), one evaluation pass and the dual sweeps on the current X^t
  const bool use_gap = pa.gap_tol > 0.0;
  const int64_t gap_every = pa.gap_every > 0 ? pa.gap_every : L;
  int64_t next_gap = -1;
  int stop = 0;
  double gap = NAN;
  for (;;) {
    int rc = run_graph(ctx, 1, L);
    if (rc) return rc;
    if ((rc = poll(ctx))) return rc;
    if (ctx->host_dev->done) break;
    if (use_gap && ctx->host_dev->t >= next_gap) {
      double ob[LAMP_OBJECTIVE_SLOTS];
      if ((rc = objective_values(ctx, ob))) return rc;
      gap = ob[9];
      if (gap <= pa.gap_tol) {
        stop = LAMP_STOP_GAP;
        break;
      }
      next_gap = ctx->host_dev->t + gap_every;
      CK(arm());  // the evaluation passes leave the device loop stopped
    }
  }
  const DevState& hd = *ctx->host_dev;
  if (stop == 0 && hd.status == 0) {
    // the device's rule (k_col_fin): infeasibility, and for eta > 0 the kappa condition
    const bool rule = hd.t >= 1 && hd.res <= pa.tol &&
                      (ctx->k.eta == 0.0 || ctx->k.infeas_only || 1.0 - hd.kappa * ctx->k.eta <= pa.tol);
    stop = rule ? LAMP_STOP_INFEAS : LAMP_STOP_MAX_ITER;
  }
  const double rule_res = hd.res;  // the infeasibility the stopping rule saw
  if (stop != LAMP_STOP_GAP && ctx->k.shared_shift && hd.status == 0) {
    // the regular iterations of the packed direct-form sweeps leave <C, X^t> out: one
    // evaluation pass of the final state provides it (its column sums may differ from the
    // iteration's in the last bits; the result keeps the value the stopping rule used)
    int rc = evaluate(ctx);
    if (rc) return rc;
    ctx->host_dev->res = rule_res;
  }
  fill_result(ctx, out, stop, gap);
  const DevState& d = *ctx->host_dev;
  if (d.status == LAMP_E_TIMEOUT) {
    if (out) out->status = LAMP_E_TIMEOUT;
    return fail(ctx, LAMP_E_TIMEOUT, "a device-side wait ran out of its iteration budget at iteration %lld",
                (long long)d.t);
  }
  if (d.status != 0) {
    if (out) out->status = LAMP_E_NUMERIC;
    return fail(ctx, LAMP_E_NUMERIC, "non-finite or out-of-range sum at iteration %lld", (long long)d.t);
  }
  if (stop == LAMP_STOP_MAX_ITER) {
    if (out) out->status = LAMP_E_NOT_CONVERGED;
    return fail(ctx, LAMP_E_NOT_CONVERGED, "max_iter reached (t=%lld, infeasibility %.3e)", (long long)d.t, d.res);
  }
  return LAMP_OK;
}

extern "C" int lamp_iterate(lamp_ctx* ctx, int64_t iters) {
  if (!ctx) return fail(nullptr, LAMP_E_INVALID, "lamp_iterate: null context");
  if (iters < 0) return fail(ctx, LAMP_E_INVALID, "iters must be >= 0");
  if (iters == 0) return LAMP_OK;
  k_ctrl<<<1, 1, 0, ctx->stream>>>(ctx->w.dev, 0, -1.0, 0, iters, 0);
  CK(cudaGetLastError());
  const int64_t L = ctx->params.check_every;
  int64_t left = iters;
  while (left >= L && L > 1) {
    int rc = run_graph(ctx, 1, L);
    if (rc) return rc;
    left -= L;
  }
  while (left > 0) {
    int rc = run_graph(ctx, 0, 1);
    if (rc) return rc;
    --left;
  }
  return LAMP_OK;
}

static int evaluate(lamp_ctx* ctx) {
  k_ctrl<<<1, 1, 0, ctx->stream>>>(ctx->w.dev, 1, -1.0, 0, 0, 0);
  CK(cudaGetLastError());
  int rc = run_graph(ctx, 2, 1);
  if (rc) return rc;
  return poll(ctx);
}

// the gradient passes need the row weights, column data and col(X^t) of the current state:
// when the last pass of the device loop (a stopped solve, lamp_objective) already evaluated
// this X^t and nothing changed the state since (lamp_set_state resets t_eval), they are in
// place and the evaluation pass is skipped
static int evaluate_if_stale(lamp_ctx* ctx) {
  int rc = poll(ctx);
  if (rc) return rc;
  const DevState& d = *ctx->host_dev;
  if (d.t_eval == d.t && d.status == 0 && d.kappa_eval == d.kappa) return LAMP_OK;
  return evaluate(ctx);
}

// run evaluation passes outside the iteration after an evaluate(): the sweeps return at
// once while dev->done is set, so clear it for the passes and set it again after
static int begin_passes(lamp_ctx* ctx) {
  k_ctrl<<<1, 1, 0, ctx->stream>>>(ctx->w.dev, 1, -1.0, 0, 0, 0);
  CK(cudaGetLastError());
  return LAMP_OK;
}
static int end_passes(lamp_ctx* ctx) {
  k_mark_done<<<1, 1, 0, ctx->stream>>>(ctx->w.dev);
  CK(cudaGetLastError());
  return LAMP_OK;
}

// widen rowpart / colpart to `width` values per point (per split); the captured graphs hold
// the old pointers, so they are dropped and rebuilt on their next use
static int ensure_part_width(lamp_ctx* ctx, int width) {
  if (width <= ctx->part_width) return LAMP_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  for (double* old : {ctx->w.rowpart, ctx->w.colpart}) {
    auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), (void*)old);
    if (it != ctx->allocs.end()) ctx->allocs.erase(it);
    cudaFree(old);
  }
  ctx->w.rowpart = ctx->w.colpart = nullptr;
  for (int s = 0; s < 3; ++s) {
    if (ctx->gexec[s]) cudaGraphExecDestroy(ctx->gexec[s]);
    ctx->gexec[s] = nullptr;
    ctx->glen[s] = 0;
  }
  int rc = dalloc(ctx, &ctx->w.rowpart, (size_t)ctx->g.rows_split * width * ctx->k.n);
  if (!rc) rc = dalloc(ctx, &ctx->w.colpart, (size_t)ctx->g.cols_split * width * ctx->k.m);
  if (rc) return rc;
  ctx->part_width = width;
  return LAMP_OK;
}

extern "C" int lamp_apply_map(lamp_ctx* ctx, const float* V, int64_t k, float* out, int side) {
  if (!ctx || !V || !out) return fail(ctx, LAMP_E_INVALID, "lamp_apply_map: null argument");
  if (k < 1 || k > 8) return fail(ctx, LAMP_E_INVALID, "lamp_apply_map: 1 <= k <= 8 value columns (got %lld)",
                                  (long long)k);
  if (side != 0 && side != 1) return fail(ctx, LAMP_E_INVALID, "lamp_apply_map: side must be 0 (p V) or 1 (p^T U)");
  int rc = ensure_part_width(ctx, (int)k);
  if (rc) return rc;
  rc = evaluate(ctx);
  if (rc) return rc;
  CK(launch_map(ctx->in, ctx->k, ctx->w, ctx->g, ctx->host_dev->cur, V, (int)k, out, side, ctx->stream));
  return LAMP_OK;
}

static int dual_values(lamp_ctx* ctx, double out[2]) {
  // evaluate() or poll() has run: host_dev->cur is the state's parity
  const int cur = ctx->host_dev->cur;
  int rc = begin_passes(ctx);
  if (rc) return rc;
  for (int which = 0; which < 2; ++which)
    CK(launch_dual(ctx->in, ctx->k, ctx->w, ctx->g, ctx->prec, cur, which, ctx->w.scratch + 4 + 2 * which,
                   ctx->stream));
  if ((rc = end_passes(ctx))) return rc;
  double h[4];
  CK(cudaMemcpyAsync(h, ctx->w.scratch + 4, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const Consts& k = ctx->k;
  // D(phi) = sum_i r_i rowmin_i - 2K <c, phi>  (eta > 0: softmin, and the constant -eta H(r))
  for (int which = 0; which < 2; ++which)
    out[which] = h[2 * which] - 2.0 * k.K * h[2 * which + 1] - (k.eta > 0.0 ? k.eta * ctx->Hr : 0.0);
  return LAMP_OK;
}

extern "C" int lamp_dual(lamp_ctx* ctx, double out[2]) {
  if (!ctx || !out) return fail(ctx, LAMP_E_INVALID, "lamp_dual: null argument");
  int rc = poll(ctx);
  if (rc) return rc;
  return dual_values(ctx, out);
}

extern "C" int lamp_round(lamp_ctx* ctx, double out[4], double* y, double* delta_r, double* delta_c) {
  if (!ctx || !out) return fail(ctx, LAMP_E_INVALID, "lamp_round: null argument");
  int rc = evaluate(ctx);
  if (rc) return rc;
  const int cur = ctx->host_dev->cur;
  if ((rc = begin_passes(ctx))) return rc;
  CK(launch_round(ctx->in, ctx->k, ctx->w, ctx->g, ctx->prec, cur, ctx->w.scratch, y, delta_r, delta_c,
                  ctx->stream));
  if ((rc = end_passes(ctx))) return rc;
  CK(cudaMemcpyAsync(out, ctx->w.scratch, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LAMP_OK;
}

extern "C" int lamp_objective(lamp_ctx* ctx, double out[LAMP_OBJECTIVE_SLOTS]) {
  if (!ctx || !out) return fail(ctx, LAMP_E_INVALID, "lamp_objective: null argument");
  return objective_values(ctx, out);
}

// the quantities of lamp_objective for the current state (one evaluation pass, then the
// dual sweeps); leaves the device loop stopped (dev->done set)
static int objective_values(lamp_ctx* ctx, double* out) {
  int rc = evaluate(ctx);
  if (rc) return rc;
  const DevState& d = *ctx->host_dev;
  const Consts& k = ctx->k;
  // H(X) = H(r) + kappa <C,X> + 2 K kappa <col(X), nu> + <r, log Z>  (App. D identity, any kappa)
  double H = ctx->Hr + d.kappa * d.costA + 2.0 * k.K * d.kappa * d.colnu + d.rlogZ;
  out[0] = d.costA;
  out[1] = d.res;
  out[2] = 0.0;  // row(X^t) = r by construction of p^{eta}(nu) (Eq. row_feasible)
  out[3] = H;
  out[4] = d.costA + 2.0 * k.K * d.res - k.eta * H;
  out[5] = (k.eta == 0.0 && d.t >= 1) ? 4.0 * k.K * d.res + 2.0 * k.K * ctx->log_m / (double)d.t : NAN;
  out[7] = k.K;
  out[8] = d.costA - k.eta * H;  // <C, X^t> - eta H(X^t)  (Eq. prob:primal_eot)
  out[9] = NAN;
  if (d.status == LAMP_E_TIMEOUT) return fail(ctx, LAMP_E_TIMEOUT, "a device-side wait ran out of its budget");
  if (d.status != 0) return fail(ctx, LAMP_E_NUMERIC, "non-finite or out-of-range sum");
  // the dual bound at theta^t and nu^t (the larger is reported)
  double D2[2];
  if ((rc = dual_values(ctx, D2))) return rc;
  out[6] = std::max(D2[0], D2[1]);
  out[9] = out[4] - out[6];  // primal-dual gap of the saddle problem (App. E.2 termination)
  return LAMP_OK;
}

static inline int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

// the envelope gradient on tensor cores: one fused recompute pass per side (S = x.y^T by
// MMA, P = 2^v w in the epilogue, P.Y by a second MMA), then a float-float finalize
static int grad_tc(lamp_ctx* ctx, float* dx, float* dy) {
  const Consts& k = ctx->k;
  const int64_t n_pad = tc_pad(k.n), m_pad = tc_pad(k.m);
  const int64_t wave = (int64_t)ctx->g.sms * 2;  // two CTAs per SM
  // every split writes 64 float32 partials per point: splits cost 1 % of a wave each here
  // (0.2 % for the sweeps), which keeps their number near the smallest that fills the waves
  const int sx = choose_split(cdiv64(k.n, tcg_tile_fixed()), cdiv64(k.m, tcg_tile_stream()), wave, 4, 0.01);
  const int sy = choose_split(cdiv64(k.m, tcg_tile_fixed()), cdiv64(k.n, tcg_tile_stream()), wave, 4, 0.01);
  int rc;
  if (!ctx->xT) {
    CK(tcg_prepare());
    if ((rc = dalloc(ctx, reinterpret_cast<uint16_t**>(&ctx->xT), (size_t)n_pad * 64))) return rc;
    if ((rc = dalloc(ctx, reinterpret_cast<uint16_t**>(&ctx->yT), (size_t)m_pad * 64))) return rc;
    CK(tc_make_map2(ctx->map_xT, ctx->xT, n_pad, 64, 64, 64));
    CK(tc_make_map2(ctx->map_yT, ctx->yT, m_pad, 64, 64, 64));
    ctx->tcg_fresh = false;
  }
  // the two sides run concurrently (dx on the context's stream, dy on a side stream), each
  // with partials of its own: one side's tail overlaps the other side's start
  const size_t need_x = (size_t)sx * k.n * 64, need_y = (size_t)sy * k.m * 64;
  const size_t need = need_x + need_y;
  if (!ctx->gside) {
    if (cudaStreamCreateWithFlags(&ctx->gside, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->gfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->gjoin, cudaEventDisableTiming) != cudaSuccess)
      return fail(ctx, LAMP_E_CUDA, "lamp_grad: stream / event creation failed");
  }
  if (need > ctx->tcg_part_floats) {
    if (ctx->tcg_part) {
      CK(cudaStreamSynchronize(ctx->stream));
      auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), (void*)ctx->tcg_part);
      if (it != ctx->allocs.end()) ctx->allocs.erase(it);
      cudaFree(ctx->tcg_part);
      ctx->tcg_part = nullptr;
      ctx->tcg_part_floats = 0;
    }
    if ((rc = dalloc(ctx, &ctx->tcg_part, need))) return rc;
    ctx->tcg_part_floats = need;
  }
  if (!ctx->tcg_fresh) {
    CK(tcg_transpose(ctx->xb, n_pad, ctx->xT, ctx->stream));
    CK(tcg_transpose(ctx->yb, m_pad, ctx->yT, ctx->stream));
    ctx->tcg_fresh = true;
  }
  if ((rc = evaluate_if_stale(ctx))) return rc;
  const int cur = ctx->host_dev->cur;
  cudaStream_t sy_st = dx ? ctx->gside : ctx->stream;
  if (dx && dy) {
    CK(cudaEventRecord(ctx->gfork, ctx->stream));
    CK(cudaStreamWaitEvent(sy_st, ctx->gfork, 0));
  }
  if (dx) {
    CK(tcg_launch(true, ctx->map_x, ctx->map_y64, ctx->map_yT, ctx->w, k, sx, ctx->tcg_part, ctx->stream));
    CK(tcg_finalize(true, ctx->tcg_part, sx, ctx->w, k, ctx->in.x, ctx->in.r, ctx->w.g2row, dx, ctx->stream));
  }
  if (dy) {
    float* party = ctx->tcg_part + need_x;
    CK(tcg_launch(false, ctx->map_y, ctx->map_x64, ctx->map_xT, ctx->w, k, sy, party, sy_st));
    CK(tcg_finalize(false, party, sy, ctx->w, k, ctx->in.y, ctx->in.r, ctx->w.colq[cur], dy, sy_st));
  }
  if (dx && dy) {
    CK(cudaEventRecord(ctx->gjoin, sy_st));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->gjoin, 0));
  }
  return LAMP_OK;
}

extern "C" int lamp_grad(lamp_ctx* ctx, float* dx, float* dy) {
  if (!ctx) return fail(nullptr, LAMP_E_INVALID, "lamp_grad: null context");
  if (ctx->pub_kind != LAMP_COST_SQEUCLID) return fail(ctx, LAMP_E_UNSUPPORTED, "lamp_grad needs LAMP_COST_SQEUCLID");
  if (ctx->prec == LAMP_PREC_BF16_TC) return grad_tc(ctx, dx, dy);
  // d > 8: the gradient is computed in chunks of 8 coordinates (partials of 8 values per point)
  int rc = ensure_part_width(ctx, std::min<int>((int)ctx->k.d, 8));
  if (rc) return rc;
  rc = evaluate_if_stale(ctx);
  if (rc) return rc;
  CK(launch_grad(ctx->in, ctx->k, ctx->w, ctx->g, ctx->prec, dx, dy, ctx->stream));
  return LAMP_OK;
}

extern "C" int lamp_get_state(lamp_ctx* ctx, double* nu, double* theta, double* logZ, double* kappa, int64_t* t,
                              float* row_shifts) {
  if (!ctx) return fail(nullptr, LAMP_E_INVALID, "lamp_get_state: null context");
  int rc = poll(ctx);
  if (rc) return rc;
  const DevState& d = *ctx->host_dev;
  const int cur = d.cur;
  if (nu) CK(cudaMemcpyAsync(nu, ctx->w.nu[cur], ctx->k.m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (theta)
    CK(cudaMemcpyAsync(theta, ctx->w.theta[cur], ctx->k.m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (logZ) CK(cudaMemcpyAsync(logZ, ctx->w.logZ, ctx->k.n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (row_shifts)
    CK(cudaMemcpyAsync(row_shifts, ctx->w.rowshift[cur], ctx->k.n * sizeof(float2), cudaMemcpyDeviceToHost,
                       ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (logZ && d.t_eval != d.t)
    for (int64_t i = 0; i < ctx->k.n; ++i) logZ[i] = NAN;
  if (kappa) *kappa = d.kappa;
  if (t) *t = d.t;
  return LAMP_OK;
}

extern "C" int lamp_set_state(lamp_ctx* ctx, const double* nu, const double* theta, double kappa, int64_t t,
                              const float* row_shifts) {
  if (!ctx || !nu || !theta) return fail(ctx, LAMP_E_INVALID, "lamp_set_state: null argument");
  if (!(kappa >= 0.0) || !std::isfinite(kappa) || t < 0) return fail(ctx, LAMP_E_INVALID, "bad kappa or t");
  for (int64_t j = 0; j < ctx->k.m; ++j)
    if (!(std::fabs(nu[j]) < 1.0) || !(std::fabs(theta[j]) < 1.0))
      return fail(ctx, LAMP_E_INVALID, "nu and theta must lie in (-1, 1)");
  int rc = poll(ctx);
  if (rc) return rc;
  const int cur = ctx->host_dev->cur;
  CK(cudaMemcpyAsync(ctx->w.nu[cur], nu, ctx->k.m * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->w.theta[cur], theta, ctx->k.m * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  k_set_state<<<1, 1, 0, ctx->stream>>>(ctx->w.dev, t, kappa);
  CK(cudaGetLastError());
  if (row_shifts) {
    for (int64_t i = 0; i < 2 * ctx->k.n; ++i)
      if (!std::isfinite(row_shifts[i])) return fail(ctx, LAMP_E_INVALID, "row_shifts must be finite");
    CK(launch_init_state(ctx->in, ctx->k, ctx->w, 0, ctx->stream));
    if (ctx->k.shared_shift) {
      // both streams use stream A's shift: keep the pairs consistent whatever was passed
      std::vector<float> rs(row_shifts, row_shifts + 2 * ctx->k.n);
      for (int64_t i = 0; i < ctx->k.n; ++i) rs[2 * i + 1] = rs[2 * i];
      CK(cudaMemcpyAsync(ctx->w.rowshift[cur], rs.data(), ctx->k.n * sizeof(float2), cudaMemcpyHostToDevice,
                         ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    } else {
      CK(cudaMemcpyAsync(ctx->w.rowshift[cur], row_shifts, ctx->k.n * sizeof(float2), cudaMemcpyHostToDevice,
                         ctx->stream));
    }
  } else if ((rc = prime(ctx))) {
    return rc;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return LAMP_OK;
}

extern "C" int lamp_step_host(lamp_ctx* ctx, const float* C_or_x, const float* y, const double* r, const double* c,
                              int64_t iters, double* infeas_out, double* nu_out) {
  if (!ctx) return fail(nullptr, LAMP_E_INVALID, "lamp_step_host: null context");
  if (!ctx->owned) return fail(ctx, LAMP_E_INVALID, "lamp_step_host needs a context from lamp_create_owned");
  const Consts& k = ctx->k;
  if (!C_or_x || !r || !c || (k.kind == COST_SQEUCLID && !y)) return fail(ctx, LAMP_E_INVALID, "null input");
  size_t na = k.kind == COST_DENSE ? (size_t)k.n * k.m : (size_t)k.n * k.d;
  CK(cudaMemcpyAsync(ctx->own_a, C_or_x, na * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  if (k.kind == COST_SQEUCLID)
    CK(cudaMemcpyAsync(ctx->own_b, y, (size_t)k.m * k.d * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->own_r, r, k.n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->own_c, c, k.m * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  const float* px = ctx->own_a;
  const float* py = ctx->own_b;
  if (ctx->pub_kind == LAMP_COST_COSINE) {
    // the same normalisation as at creation (the data describe the same problem)
    CK(launch_unit_rows(ctx->own_a, k.n, k.d, ctx->xn, reinterpret_cast<unsigned int*>(ctx->w.scratch),
                        ctx->stream));
    CK(launch_unit_rows(ctx->own_b, k.m, k.d, ctx->yn, reinterpret_cast<unsigned int*>(ctx->w.scratch),
                        ctx->stream));
    px = ctx->xn;
    py = ctx->yn;
  }
  if (ctx->prec == LAMP_PREC_BF16_TC) {
    CK(tc_convert(px, k.n, k.d, ctx->xr, ctx->xb, ctx->stream));
    CK(tc_convert(py, k.m, k.d, ctx->yr, ctx->yb, ctx->stream));
    ctx->tcg_fresh = false;  // the gradient pass transposes the new points on its next call
  }
  int rc = lamp_iterate(ctx, iters);
  if (rc) return rc;
  CK(cudaMemcpyAsync(&ctx->host_dev->res, &ctx->w.dev->res, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (nu_out) {
    // the buffer parity is only known on the device; copy both halves' candidate after reading cur
    CK(cudaMemcpyAsync(&ctx->host_dev->cur, &ctx->w.dev->cur, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpyAsync(nu_out, ctx->w.nu[ctx->host_dev->cur], k.m * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (infeas_out) *infeas_out = ctx->host_dev->res;
  return LAMP_OK;
}

extern "C" int lamp_time_kernels(lamp_ctx* ctx, int64_t iters, double* ms_out) {
  if (!ctx || !ms_out) return fail(ctx, LAMP_E_INVALID, "lamp_time_kernels: null argument");
  if (iters < 1 || iters > 1000) return fail(ctx, LAMP_E_INVALID, "iters must be in [1, 1000]");
  k_ctrl<<<1, 1, 0, ctx->stream>>>(ctx->w.dev, 0, -1.0, 0, iters + 1, 0);
  CK(cudaGetLastError());
  // one untimed iteration first, then all timed launches back to back with an event
  // between consecutive kernels; a single synchronisation at the end, so no launch
  // latency of an idle stream falls inside a kernel's interval
  std::vector<cudaEvent_t> ev((size_t)(4 * iters + 1), nullptr);
  int rc = LAMP_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = fail(ctx, LAMP_E_CUDA, "cudaEventCreate failed");
  for (int part = 0; part < 4 && rc == LAMP_OK; ++part) {
    cudaError_t e = launch_iteration_part(ctx->in, ctx->k, ctx->w, ctx->g, ctx->prec, part, 0, ctx->stream);
    if (e != cudaSuccess) rc = fail(ctx, LAMP_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  }
  if (rc == LAMP_OK) cudaEventRecord(ev[0], ctx->stream);
  for (int64_t it = 0; it < iters && rc == LAMP_OK; ++it) {
    for (int part = 0; part < 4; ++part) {
      cudaError_t e = launch_iteration_part(ctx->in, ctx->k, ctx->w, ctx->g, ctx->prec, part, 0, ctx->stream);
      if (e != cudaSuccess) {
        rc = fail(ctx, LAMP_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
        break;
      }
      cudaEventRecord(ev[(size_t)(4 * it + part + 1)], ctx->stream);
    }
  }
  double acc[4] = {0, 0, 0, 0};
  if (rc == LAMP_OK) {
    cudaError_t e = cudaEventSynchronize(ev.back());
    if (e != cudaSuccess) rc = fail(ctx, LAMP_E_CUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
  }
  for (int64_t it = 0; it < iters && rc == LAMP_OK; ++it)
    for (int part = 0; part < 4; ++part) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[(size_t)(4 * it + part)], ev[(size_t)(4 * it + part + 1)]);
      acc[part] += ms;
    }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (rc) return rc;
  for (int part = 0; part < 4; ++part) ms_out[part] = acc[part] / (double)iters;
  return LAMP_OK;
}

extern "C" int64_t lamp_launches_per_iteration(const lamp_ctx* ctx) {
  if (!ctx) return 0;
  return launches_per_iteration(ctx->k, ctx->prec);
}

extern "C" int lamp_selftest_wait_timeout(int64_t polls, int* status) {
  if (!status || polls < 1 || polls > (int64_t)1 << 30)
    return fail(nullptr, LAMP_E_INVALID, "lamp_selftest_wait_timeout: status must be non-NULL, 1 <= polls <= 2^30");
  int rc = tc_wait_selftest((uint32_t)polls, status);
  if (rc) return fail(nullptr, rc, "lamp_selftest_wait_timeout: CUDA error");
  return LAMP_OK;
}

extern "C" const char* lamp_last_error(const lamp_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

extern "C" void lamp_destroy(lamp_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (int s = 0; s < 3; ++s)
    if (ctx->gexec[s]) cudaGraphExecDestroy(ctx->gexec[s]);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->host_dev) cudaFreeHost(ctx->host_dev);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  if (ctx->gside) {
    cudaStreamSynchronize(ctx->gside);
    cudaStreamDestroy(ctx->gside);
  }
  if (ctx->gfork) cudaEventDestroy(ctx->gfork);
  if (ctx->gjoin) cudaEventDestroy(ctx->gjoin);
  delete ctx;
}
