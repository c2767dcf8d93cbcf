// lamp_marginals_noalloc: the marginal evaluation pass (row log-normalisers,
// column sums and <C, X> of X = diag(r) p^{1/kappa}(nu)) with every piece of
// scratch memory taken from one statically sized device array that ships with
// the library, so that the call itself allocates nothing.
//
// Who needs this: callers that are not allowed to call cudaMalloc where they
// run.  A plugin executed by a host framework that owns all device memory
// through its own pool (an inference server's execute callback, a fixed
// memory budget handed out up front) cannot take memory behind the pool's
// back, and cudaMalloc / cudaFree can synchronise the device, which a
// latency-bound caller cannot afford in its hot loop.  The regular entry
// points allocate a context workspace in lamp_create; this one does not.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its kScratchBytes until the process exits.  Host code cannot
// use the variable's name as a device pointer (in host code it names a host
// shadow), so the first call on each device, with that device current, looks
// up the real address with cudaGetSymbolAddress and caches it per device,
// together with the device's current CUDA context.  A call that finds another
// context current on that device (the primary context was reset or torn down
// and re-created, which reloads the module and can move the array) looks the
// address up again.  Make the first call on a device, and the first call after
// such a reset, before any stream capture is started.
//
// All calls on a device share the one array and leave their contents in it;
// the call clears what must start at zero.  Calls whose GPU work overlaps
// (different streams, or different host threads) race on the array and
// corrupt each other: issue them on one stream, one after the other.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/lamp.h"
#include "lamp_common.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};  // the context the cached address belongs to
std::mutex g_scratch_mu;

// the calling thread's current CUDA context (driver API, looked up once through the
// runtime's entry-point query so that the library needs no link to libcuda)
cudaError_t current_context(void** out) {
  typedef int (*CtxGetCurrentFn)(void**);
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<CtxGetCurrentFn>(p);
  }
  *out = nullptr;
  return fn(out) == 0 ? cudaSuccess : cudaErrorIncompatibleDriverContext;
}

int noalloc_fail(int code, const char* msg) {
  lamp::set_last_error_null(msg);
  return code;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// sequential carve-out of the scratch array; returns the bytes a layout needs
struct Carver {
  unsigned char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + off);
    off += align256(std::max<size_t>(count, 1) * sizeof(T));
    return p;
  }
};

__global__ void k_noalloc_init(lamp::DevState* dev, double kappa, const double* __restrict__ nu_in,
                               double* __restrict__ nu0, double* __restrict__ th0, int64_t m) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) {
    dev->t = 0;
    dev->kappa = kappa;
    dev->swf_kap = -1.0;
    dev->cur = 0;
    dev->done = 0;
    dev->status = 0;
    dev->eval_only = 1;
    dev->tol = -1.0;
    dev->tmax = 0;
    dev->ticket = 0u;
    dev->t_eval = -1;
  }
  if (j < m) {
    nu0[j] = nu_in[j];
    th0[j] = 0.0;
  }
}

// <C, X> to the caller; NaN when a row sum fell outside the representable range
__global__ void k_noalloc_out(const lamp::DevState* dev, double* cost_out) {
  *cost_out = dev->status == 0 ? dev->costA : nan("");
}

}  // namespace

extern "C" int lamp_marginals_noalloc(const lamp_problem* prob, double K, double kappa, const double* nu,
                                      double* logZ_out, double* col_out, double* cost_out, void* stream) {
  using namespace lamp;
  if (!prob || !nu || !logZ_out || !col_out) return noalloc_fail(LAMP_E_INVALID, "null argument");
  if (prob->n < 1 || prob->m < 1) return noalloc_fail(LAMP_E_INVALID, "n and m must be >= 1");
  if (prob->kind >= LAMP_COST_L1 && prob->kind <= LAMP_COST_COSINE)
    return noalloc_fail(LAMP_E_UNSUPPORTED, "lamp_marginals_noalloc supports LAMP_COST_DENSE and LAMP_COST_SQEUCLID");
  if (prob->kind != LAMP_COST_DENSE && prob->kind != LAMP_COST_SQEUCLID)
    return noalloc_fail(LAMP_E_INVALID, "unknown cost kind");
  if (!prob->r || !prob->c) return noalloc_fail(LAMP_E_INVALID, "r and c must be non-null");
  if (prob->kind == LAMP_COST_DENSE && (!prob->C || prob->ldc < prob->m))
    return noalloc_fail(LAMP_E_INVALID, "DENSE needs C with ldc >= m");
  if (prob->kind == LAMP_COST_SQEUCLID) {
    if (!prob->x || !prob->y) return noalloc_fail(LAMP_E_INVALID, "SQEUCLID needs x and y");
    if (prob->d < 1) return noalloc_fail(LAMP_E_INVALID, "d must be >= 1");
    if (prob->d > 8) return noalloc_fail(LAMP_E_UNSUPPORTED, "the allocation-free variant supports d <= 8");
    if (!(prob->cost_scale > 0.0) || !std::isfinite(prob->cost_scale))
      return noalloc_fail(LAMP_E_INVALID, "cost_scale must be given (> 0)");
  }
  if (!(K > 0.0) || !std::isfinite(K)) return noalloc_fail(LAMP_E_INVALID, "K must be > 0");
  if (!(kappa >= 0.0) || !std::isfinite(kappa)) return noalloc_fail(LAMP_E_INVALID, "kappa must be >= 0");

  int devi = 0;
  if (cudaGetDevice(&devi) != cudaSuccess || devi < 0 || devi >= kMaxDevices)
    return noalloc_fail(LAMP_E_CUDA, "cudaGetDevice failed");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    // the runtime makes the device's primary context current on first use; the symbol
    // lookup below does that too, so query the context after it when nothing is cached
    void* ctx = nullptr;
    cudaError_t e = current_context(&ctx);
    if (e != cudaSuccess) return noalloc_fail(LAMP_E_CUDA, "cuCtxGetCurrent failed");
    if (!g_scratch_addr[devi] || !ctx || ctx != g_scratch_ctx[devi]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        char msg[160];
        std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return noalloc_fail(LAMP_E_CUDA, msg);
      }
      if (current_context(&ctx) != cudaSuccess || !ctx) return noalloc_fail(LAMP_E_CUDA, "cuCtxGetCurrent failed");
      g_scratch_addr[devi] = p;
      g_scratch_ctx[devi] = ctx;
    }
    base = g_scratch_addr[devi];
  }
  cudaStream_t st = (cudaStream_t)stream;

  Consts k{};
  k.n = prob->n;
  k.m = prob->m;
  k.d = prob->kind == LAMP_COST_SQEUCLID ? (int32_t)prob->d : 0;
  k.kind = prob->kind;
  k.zdot = 0;  // direct form only (dense, or |x - y|^2 with d <= 8)
  k.K = K;
  k.s = prob->kind == LAMP_COST_SQEUCLID ? prob->cost_scale : 1.0;
  k.tau1 = k.tau2 = 1.0 / (2.0 * K);
  k.eta = 0.0;
  k.alpha = 0.01;
  k.alpha_m = 0.01 / (double)k.m;
  k.clipb = std::tanh(0.55);
  k.W = 5.0 * K;
  k.rnx = 0.0;

  prepare_kernels();
  Geometry g{};
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devi) != cudaSuccess || sms < 1)
      return noalloc_fail(LAMP_E_CUDA, "cudaDeviceGetAttribute failed");
    g.sms = sms;
    const int prec = LAMP_PREC_FP32;
    int64_t to = (k.n + tile_outer(k, prec) - 1) / tile_outer(k, prec);
    int64_t ti = (k.m + tile_inner(k, prec) - 1) / tile_inner(k, prec);
    int64_t tco = (k.m + tile_outer_cols(k, prec) - 1) / tile_outer_cols(k, prec);
    int64_t tci = (k.n + tile_inner_cols(k, prec) - 1) / tile_inner_cols(k, prec);
    // at most 4 splits per sweep keeps the scratch layout small
    auto pick = [&](int64_t tout, int64_t tin, int64_t wave) {
      int best = 1;
      double bs = -1.0;
      for (int s = 1; s <= 4 && s <= std::max<int64_t>(tin, 1); ++s) {
        int64_t ctas = tout * s, waves = (ctas + wave - 1) / wave;
        double sc = (double)ctas / (double)(waves * wave) - 0.002 * s;
        if (sc > bs + 1e-12) { bs = sc; best = s; }
      }
      return best;
    };
    g.rows_tiles = (int)to;
    g.cols_tiles = (int)tco;
    g.rows_split = pick(to, ti, (int64_t)sms * sweep_blocks_per_sm(k, prec, 0));
    g.cols_split = pick(tco, tci, (int64_t)sms * sweep_blocks_per_sm(k, prec, 1));
  }

  // carve the workspace out of the static array
  const size_t n = (size_t)k.n, m = (size_t)k.m;
  Carver cv{reinterpret_cast<unsigned char*>(base)};
  Work w{};
  for (int b = 0; b < 2; ++b) {
    w.nu[b] = cv.take<double>(m);
    w.theta[b] = cv.take<double>(m);
    w.colq[b] = cv.take<float4>(m);
    w.rowshift[b] = cv.take<float2>(n);
  }
  w.g2row = cv.take<float4>(n);
  w.rowpart = cv.take<double>((size_t)g.rows_split * 2 * n);
  w.colpart = cv.take<double>((size_t)g.cols_split * 3 * m);
  w.nx = cv.take<double>(n);
  w.ny = cv.take<double>(m);
  w.rowred = cv.take<double>((size_t)fin_blocks(k.n));
  w.colred = cv.take<double>(3 * (size_t)fin_blocks(k.m));
  w.rowmax = cv.take<float>((size_t)g.rows_split * 2 * n);
  w.scratch = cv.take<double>(1);
  w.dev = cv.take<DevState>(1);
  w.logZ = logZ_out;
  w.colA = col_out;
  if (cv.off > kScratchBytes) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "n=%lld, m=%lld need %zu bytes of scratch; the static array holds %zu (about 136 n + 168 m bytes "
                  "must fit)",
                  (long long)k.n, (long long)k.m, cv.off, kScratchBytes);
    return noalloc_fail(LAMP_E_INVALID, msg);
  }

  Inputs in{};
  in.C = prob->C;
  in.ldc = prob->ldc;
  in.x = prob->x;
  in.y = prob->y;
  in.r = prob->r;
  in.c = prob->c;

  k_noalloc_init<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(w.dev, kappa, nu, w.nu[0], w.theta[0], k.m);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_init_state(in, k, w, 0, st);
  if (e == cudaSuccess) e = launch_prime(in, k, w, g, LAMP_PREC_FP32, st);
  if (e == cudaSuccess) e = launch_iteration(in, k, w, g, LAMP_PREC_FP32, 1, st);
  if (e == cudaSuccess && cost_out) {
    k_noalloc_out<<<1, 1, 0, st>>>(w.dev, cost_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    char msg[160];
    std::snprintf(msg, sizeof(msg), "kernel launch: %s", cudaGetErrorString(e));
    return noalloc_fail(LAMP_E_CUDA, msg);
  }
  return LAMP_OK;
}
