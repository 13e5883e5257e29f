// The C ABI of include/cs.h: argument checks, ownership of device memory and
// the host-side order of the stream-ordered launches of one solve
// (Algorithm 1: per outer iteration one persistent Euler kernel and one refit
// kernel; then the objective and the kept trial).
#include <cmath>
#include <cstring>
#include <string>
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

struct cs_problem {
  cs::ProblemDev P;
  cs::SolveDev S;
  // timing marks: event pair k brackets launch group k of category cats[k]
  std::vector<cudaEvent_t> events;
  std::vector<int> cats;
  int n_marks = 0, n_create_marks = 0;
  bool capturing = false;     // the solve's outer loop is being captured into a graph
  int64_t submissions = 0;    // host submissions of the last solve's device work (launches outside the graph + 1)
};

namespace cs {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  static thread_local int configured_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured_device != dev) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    configured_device = dev;
  }
  return cudaMallocAsync(p, bytes, s);
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

namespace {

cs_status fail(cs_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

cs_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? CS_ENOMEM : CS_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CS_CUDA(call, what)                          \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// stream of the allocation in progress on this thread (calls on different
// problems may run on different threads at once)
thread_local cudaStream_t g_alloc_stream = nullptr;

template <typename T>
cudaError_t alloc(T** p, size_t elems) {
  return dev_alloc((void**)p, (elems == 0 ? 1 : elems) * sizeof(T), g_alloc_stream);
}

void free_solve(SolveDev& S, cudaStream_t st) {
  void* ptrs[] = {S.R, S.X0, S.X1, S.state, S.lead, S.job, S.sigma, S.energy, S.ssize, S.sidx, S.work, S.rec_c,
                  S.rec_e, S.x_hat, S.sigma_hat, S.stats, S.bar, S.err, S.singular, S.err4, S.e_hist, S.s_hist,
                  S.sig_outer, S.R_outer};
  for (void* q : ptrs) dev_free(q, st);
  S = SolveDev();
}

void free_problem(ProblemDev& P) {
  void* ptrs[] = {P.A, P.y, P.G, P.hz, P.g, P.Gs, P.Gt, P.Gt2, P.gscale, P.flag};
  for (void* q : ptrs) dev_free(q, P.stream);
  P = ProblemDev();
}

size_t compute_bytes(int precision) { return precision == CS_P_FP64 ? 8 : 4; }

// (Re)size the per-solve buffers for `trials`, n_outer and record_steps.  A
// batched solve (`pool` false) shares one refit workspace across its problems.
// Zero both X buffers: every product form relies on X rows >= N being zero,
// and the forms lay X out differently, so rows a previous solve of another
// form wrote may sit where this one keeps padding.
static cudaError_t clear_x(ProblemDev& P, SolveDev& S) {
  cudaError_t e = cudaMemsetAsync(S.X0, 0, S.x_bytes, P.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.X1, 0, S.x_bytes, P.stream);
  return e;
}

cs_status ensure_solve(ProblemDev& P, SolveDev& S, const cs_params& prm, int trials, bool pool = true) {
  const int rec = prm.record_steps > 0 ? std::min(prm.record_steps, prm.n_steps) : 0;
  const bool fits = S.R && trials <= S.cap_trials && prm.n_outer <= S.cap_outer && rec <= S.cap_record &&
                    (prm.record_outer == 0 || S.sig_outer) &&
                    compute_bytes(prm.precision) <= compute_bytes(S.cap_prec < 0 ? 0 : S.cap_prec) &&
                    (!pool || S.work);
  if (!fits) {
    free_solve(S, P.stream);
    g_alloc_stream = P.stream;
    const size_t N = (size_t)P.N, Np = (size_t)P.Npad, T = (size_t)trials;
    const size_t cb = compute_bytes(prm.precision);
    CS_CUDA(alloc(&S.R, N * T), "cudaMalloc R");
    const size_t T4 = (T + 3) / 4 * 4;
    CS_CUDA(dev_alloc(&S.X0, Np * T4 * cb, P.stream), "cudaMalloc X0");
    CS_CUDA(dev_alloc(&S.X1, Np * T4 * cb, P.stream), "cudaMalloc X1");
    S.x_bytes = Np * T4 * cb;
    CS_CUDA(alloc(&S.sigma, N * T), "cudaMalloc sigma");
    CS_CUDA(alloc(&S.energy, T), "cudaMalloc energy");
    CS_CUDA(alloc(&S.ssize, (size_t)prm.n_outer * T), "cudaMalloc ssize");
    CS_CUDA(alloc(&S.sidx, N * T), "cudaMalloc sidx");
    CS_CUDA(alloc(&S.lead, T), "cudaMalloc lead");
    CS_CUDA(alloc(&S.job, 1), "cudaMalloc job");
    CS_CUDA(dev_alloc(&S.state, 3 * N * T * cb, P.stream), "cudaMalloc state");
    if (pool) {
      S.work_blocks = (int)std::min<size_t>(T, (size_t)P.num_sms);
      S.work_stride = N * N + 4 * N;  // the refit's matrix and four vectors
      CS_CUDA(alloc(&S.work, (size_t)S.work_blocks * S.work_stride), "cudaMalloc refit workspace");
    }
    if (prm.record_outer) {
      CS_CUDA(alloc(&S.sig_outer, (size_t)prm.n_outer * N * T), "cudaMalloc outer supports");
      CS_CUDA(alloc(&S.R_outer, (size_t)prm.n_outer * N * T), "cudaMalloc outer signals");
    }
    CS_CUDA(alloc(&S.rec_c, (size_t)rec * N * T), "cudaMalloc rec_c");
    CS_CUDA(alloc(&S.rec_e, (size_t)rec * N * T), "cudaMalloc rec_e");
    CS_CUDA(alloc(&S.x_hat, N), "cudaMalloc x_hat");
    CS_CUDA(alloc(&S.sigma_hat, N), "cudaMalloc sigma_hat");
    CS_CUDA(alloc(&S.stats, CS_STATS_LEN), "cudaMalloc stats");
    CS_CUDA(alloc(&S.bar, kMaxEulerCtas + 1), "cudaMalloc publication flags");
    CS_CUDA(alloc(&S.err, 1), "cudaMalloc err");
    CS_CUDA(alloc(&S.singular, 1), "cudaMalloc singular");
    CS_CUDA(alloc(&S.err4, 4), "cudaMalloc error scratch");
    S.cap_trials = trials;
    S.cap_outer = prm.n_outer;
    S.cap_record = rec;
    S.cap_prec = prm.precision;
  }
  S.trials = trials;
  S.n_outer = prm.n_outer;
  S.record_steps = rec;
  S.precision = prm.precision;
  if (prm.readout == CS_READOUT_BEST) {
    // history of the best-configuration readout: per step the configuration
    // (N x T bytes) and each CTA's energy partials (T doubles)
    const size_t steps = (size_t)prm.n_steps + 1;
    const size_t ne = steps * (size_t)P.num_sms * trials, ns = steps * (size_t)P.N * trials;
    if (!S.e_hist || S.cap_e_hist < ne || S.cap_s_hist < ns) {
      dev_free(S.e_hist, P.stream);
      dev_free(S.s_hist, P.stream);
      S.e_hist = nullptr;
      S.s_hist = nullptr;
      S.cap_e_hist = S.cap_s_hist = 0;
      g_alloc_stream = P.stream;
      CS_CUDA(alloc(&S.e_hist, ne), "cudaMalloc readout energies");
      CS_CUDA(alloc(&S.s_hist, ns), "cudaMalloc readout configurations");
      S.cap_e_hist = ne;
      S.cap_s_hist = ns;
    }
  }
  return CS_OK;
}

cs_status check_params(const cs_params* p, int trials) {
  if (!p) return fail(CS_EINVAL, "params is NULL");
  if (trials < 1) return fail(CS_EINVAL, "trials must be >= 1");
  if (p->n_outer < 1 || p->n_steps < 1) return fail(CS_EINVAL, "n_outer and n_steps must be >= 1");
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return fail(CS_EINVAL, "dt must be > 0");
  if (!(p->tau > 0.0)) return fail(CS_EINVAL, "tau must be > 0");
  if (p->pump_kind != CS_PUMP_LINEAR && p->pump_kind != CS_PUMP_SIGMOID) return fail(CS_EINVAL, "bad pump_kind");
  if (p->pump_kind == CS_PUMP_SIGMOID && !(p->width > 0.0)) return fail(CS_EINVAL, "sigmoid width must be > 0");
  if (p->init_kind != CS_INIT_UNIFORM && p->init_kind != CS_INIT_NORMAL) return fail(CS_EINVAL, "bad init_kind");
  if (p->field != CS_FIELD_CN && p->field != CS_FIELD_BN) return fail(CS_EINVAL, "bad field");
  if (p->refit != CS_REFIT_EXACT && p->refit != CS_REFIT_JACOBI && p->refit != CS_REFIT_CG)
    return fail(CS_EINVAL, "bad refit");
  if (p->refit == CS_REFIT_CG && (p->cg_iters < 1 || !(p->cg_tol >= 0.0) || !std::isfinite(p->cg_tol)))
    return fail(CS_EINVAL, "the conjugate-gradient refit needs cg_iters >= 1 and cg_tol >= 0");
  if (p->refit == CS_REFIT_JACOBI && (!(p->jacobi_dt > 0.0) || !std::isfinite(p->jacobi_dt) || p->jacobi_iters < 1))
    return fail(CS_EINVAL, "the damped Jacobi refit needs jacobi_dt > 0 and jacobi_iters >= 1");
  if (p->precision < CS_P_FP64 || p->precision > CS_P_FP8) return fail(CS_EINVAL, "bad precision");
  if (p->eta_init > 0.0 && !(p->velo > 0.0)) return fail(CS_EINVAL, "velo must be > 0 with an eta schedule");
  if (p->record_steps < 0) return fail(CS_EINVAL, "record_steps must be >= 0");
  if (p->record_outer != 0 && p->record_outer != 1) return fail(CS_EINVAL, "record_outer must be 0 or 1");
  if (p->init_R != CS_INIT_R_ZEEMAN && p->init_R != CS_INIT_R_LASSO) return fail(CS_EINVAL, "bad init_R");
  if (p->init_R == CS_INIT_R_LASSO &&
      (p->lasso_iters < 1 || !(p->lasso_lambda >= 0.0) || !std::isfinite(p->lasso_lambda)))
    return fail(CS_EINVAL, "the LASSO initial R needs lasso_iters >= 1 and lasso_lambda >= 0");
  if (p->timeout_ms <= 0) return fail(CS_EINVAL, "timeout_ms must be > 0");
  if (p->test_phantom_ctas < 0 || p->test_phantom_ctas > 1024) return fail(CS_EINVAL, "bad test_phantom_ctas");
  if (p->cluster_size != 0 && p->cluster_size != 1 && p->cluster_size != 2 && p->cluster_size != 4 &&
      p->cluster_size != 8)
    return fail(CS_EINVAL, "cluster_size must be 0 (automatic), 1, 2, 4 or 8");
  if (p->max_ctas < 0) return fail(CS_EINVAL, "max_ctas must be >= 0");
  if (p->stream_g != 0 && p->stream_g != 1) return fail(CS_EINVAL, "stream_g must be 0 or 1");
  if (p->stream_g == 1 && p->precision == CS_P_FP64) return fail(CS_EINVAL, "FP64 G_off is never streamed");
  if (p->autotune != 0 && p->autotune != 1) return fail(CS_EINVAL, "autotune must be 0 or 1");
  if (p->tensor_form < 0 || p->tensor_form > 4) return fail(CS_EINVAL, "tensor_form must be 0, 1, 2, 3 or 4");
  if (p->tensor_form >= 2 && (p->precision == CS_P_FP64 || p->precision == CS_P_FP8))
    return fail(CS_EINVAL, "tensor_form >= 2: no tensor-core form for FP64 or FP8 storage");
  if (p->tensor_form == 4 && p->precision == CS_P_FP32 && p->stream_g == 1)
    return fail(CS_EINVAL, "tensor_form = 4: the single-problem tcgen05 form keeps FP32 G_off resident");
  if (p->self_term != 0 && p->self_term != 1) return fail(CS_EINVAL, "self_term must be 0 or 1");
  if (p->readout != CS_READOUT_FINAL && p->readout != CS_READOUT_BEST) return fail(CS_EINVAL, "bad readout");
  if (p->readout == CS_READOUT_BEST && p->field != CS_FIELD_BN)
    return fail(CS_EINVAL, "readout = CS_READOUT_BEST needs the binarised field (CS_FIELD_BN)");
  const double vals[] = {p->p0, p->p1, p->p_thr, p->d, p->t0, p->width, p->beta, p->K, p->j,
                         p->eta_init, p->eta_end, p->velo, p->init_scale};
  for (double v : vals)
    if (!std::isfinite(v)) return fail(CS_EINVAL, "non-finite parameter");
  return CS_OK;
}

// Threshold of outer iteration i (Eq. etaSchedulling), or sqrt(2 lambda) when fixed.
double eta_at(int i, const cs_params& p, double lambda) {
  if (p.eta_init <= 0.0) return std::sqrt(2.0 * lambda);
  return std::max(p.eta_init * (1.0 - i / p.velo), p.eta_end);
}

cudaError_t mark(cs_problem* p, int cat, bool begin) {
  const int k = begin ? p->n_marks : p->n_marks - 1;
  const size_t need = 2 * (size_t)(k + 1);
  while (p->events.size() < need) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    p->events.push_back(ev);
  }
  if (begin) {
    if ((int)p->cats.size() <= k) p->cats.resize(k + 1);
    p->cats[k] = cat;
    ++p->n_marks;
  }
  // (inside a stream capture the record becomes an event-record node of the graph)
  return p->capturing ? cudaEventRecordWithFlags(p->events[2 * k + (begin ? 0 : 1)], p->P.stream,
                                                 cudaEventRecordExternal)
                      : cudaEventRecord(p->events[2 * k + (begin ? 0 : 1)], p->P.stream);
}

}  // namespace

cudaStream_t problem_stream(const cs_problem* p) { return p->P.stream; }
void set_problem_stream(cs_problem* p, cudaStream_t s) { p->P.stream = s; }
int64_t problem_N(const cs_problem* p) { return p->P.N; }
int64_t problem_M(const cs_problem* p) { return p->P.M; }

RefitJob make_job(const ProblemDev& P, const SolveDev& S, const cs_params& prm) {
  RefitJob J;
  J.G = P.G;
  J.hz = P.hz;
  J.g = P.g;
  J.A = P.A;
  J.y = P.y;
  J.sigma = S.sigma;
  J.R = S.R;
  J.sidx = S.sidx;
  J.lead = S.lead;
  J.ssize = S.ssize;
  J.energy = S.energy;
  J.x_hat = S.x_hat;
  J.sigma_hat = S.sigma_hat;
  J.stats = S.stats;
  J.N = (int)P.N;
  J.M = (int)P.M;
  J.T = S.trials;
  J.lambda = P.lambda;
  J.singular = S.singular;
  J.err = S.err;
  J.refit = prm.refit;
  J.jacobi_iters = prm.jacobi_iters;
  J.jacobi_dt = prm.jacobi_dt;
  J.cg_iters = prm.cg_iters;
  J.cg_tol = prm.cg_tol;
  J.precision = prm.precision;
  J.gscale = prm.precision == CS_P_FP8 ? P.gscale : nullptr;
  return J;
}

}  // namespace cs

using namespace cs;

// Executable graphs (one per cs_solve and per cs_solve_batch) stay alive until
// they have run: each is kept with an event recorded after its launch, and the
// finished ones are destroyed at the next solve.  (The event, not the stream,
// tells: a caller may destroy its stream before the next solve.)
namespace {
std::mutex g_graph_mu;
std::vector<std::pair<cudaEvent_t, cudaGraphExec_t>> g_graphs;

void reap_graphs() {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (size_t i = 0; i < g_graphs.size();) {
    if (cudaEventQuery(g_graphs[i].first) != cudaErrorNotReady) {
      cudaGetLastError();
      cudaGraphExecDestroy(g_graphs[i].second);
      cudaEventDestroy(g_graphs[i].first);
      g_graphs[i] = g_graphs.back();
      g_graphs.pop_back();
    } else {
      ++i;
    }
  }
}

// Launch `exec` on `st` and keep it until it has run; on failure the graph is
// destroyed here.
cudaError_t launch_and_keep(cudaGraphExec_t exec, cudaStream_t st) {
  cudaError_t e = cudaGraphLaunch(exec, st);
  cudaEvent_t done = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(done, st);
  if (e != cudaSuccess) {
    // not launched, or launched without a completion event: wait for the
    // stream before destroying the graph
    cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    if (done) cudaEventDestroy(done);
    return e;
  }
  std::lock_guard<std::mutex> lk(g_graph_mu);
  g_graphs.emplace_back(done, exec);
  return cudaSuccess;
}
}  // namespace

extern "C" {

void cs_params_default(cs_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n_outer = 20;
  p->n_steps = 1000;
  p->dt = 0.01;
  p->pump_kind = CS_PUMP_LINEAR;
  p->p0 = 0.0;
  p->p1 = 1.5;
  p->p_thr = 1.0;
  p->d = 0.4;
  p->t0 = 4.0;
  p->width = 2.0;
  p->beta = 0.2;
  p->tau = 1.0;
  p->K = 1.0;
  p->j = 1.0;
  p->eta_init = 0.0;
  p->eta_end = 0.0;
  p->velo = 51.0;
  p->init_kind = CS_INIT_UNIFORM;
  p->init_scale = 0.01;
  p->field = CS_FIELD_CN;
  p->refit = CS_REFIT_EXACT;
  p->jacobi_dt = 0.1;
  p->jacobi_iters = 100;
  p->cg_iters = 10000;
  p->cg_tol = 1e-10;
  p->init_R = CS_INIT_R_ZEEMAN;
  p->lasso_iters = 500;
  p->lasso_lambda = 1e-3;
  p->precision = CS_P_FP32;
  p->seed = 0;
  p->instance = 0;
  p->record_steps = 0;
  p->timeout_ms = 10000;
}

const char* cs_last_error(void) { return g_last_error.c_str(); }

cs_status cs_problem_create(const double* A, const double* y, int64_t M, int64_t N, double lambda, int on_device,
                            void* stream, cs_problem** out) {
  if (!out) return fail(CS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!A || !y) return fail(CS_EINVAL, "A or y is NULL");
  if (M < 1 || N < 1) return fail(CS_EINVAL, "M and N must be >= 1");
  if (M > (1 << 20) || N > (1 << 16)) return fail(CS_EINVAL, "M or N too large");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(CS_EINVAL, "lambda must be finite and >= 0");
  cs_problem* p = new cs_problem();
  ProblemDev& P = p->P;
  P.M = M;
  P.N = N;
  P.Npad = (N + kPadN - 1) / kPadN * kPadN;
  P.lambda = lambda;
  P.stream = (cudaStream_t)stream;
  auto bail = [&](cs_status st) {
    free_problem(P);
    for (cudaEvent_t ev : p->events) cudaEventDestroy(ev);
    delete p;
    return st;
  };
  cudaError_t e = cudaGetDevice(&P.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, P.device);
  if (e != cudaSuccess) return bail(cuda_fail(e, "device query"));
  const size_t MN = (size_t)M * N;
  g_alloc_stream = P.stream;
  if ((e = alloc(&P.A, MN)) != cudaSuccess || (e = alloc(&P.y, (size_t)M)) != cudaSuccess ||
      (e = alloc(&P.G, (size_t)N * N)) != cudaSuccess || (e = alloc(&P.hz, (size_t)N)) != cudaSuccess ||
      (e = alloc(&P.g, (size_t)N)) != cudaSuccess || (e = alloc(&P.flag, 1)) != cudaSuccess)
    return bail(cuda_fail(e, "cudaMalloc problem"));
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if ((e = cudaMemcpyAsync(P.A, A, MN * sizeof(double), kind, P.stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(P.y, y, (size_t)M * sizeof(double), kind, P.stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(P.flag, 0, sizeof(int), P.stream)) != cudaSuccess)
    return bail(cuda_fail(e, "copy A, y"));
  if ((e = mark(p, TM_GRAM, true)) != cudaSuccess || (e = launch_gram(P)) != cudaSuccess ||
      (e = mark(p, TM_GRAM, false)) != cudaSuccess)
    return bail(cuda_fail(e, "gram launch"));
  P.launches = 2;
  p->n_create_marks = p->n_marks;
  int flag = 0;
  if ((e = cudaMemcpyAsync(&flag, P.flag, sizeof(int), cudaMemcpyDeviceToHost, P.stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(P.stream)) != cudaSuccess)
    return bail(cuda_fail(e, "gram"));
  if (flag) return bail(fail(CS_EINVAL, "A or y has a non-finite value"));
  *out = p;
  return CS_OK;
}

// The outer loop of Algorithm 1 for one problem (every CIM run, readout,
// refit and recording) and the final objective and selection, queued on
// P.stream (the capture stream while cs_solve captures them into its graph).
static cs_status queue_outer_loop(cs_problem* p, const cs_params* prm, long long timeout_cycles) {
  ProblemDev& P = p->P;
  SolveDev& S = p->S;
  for (int i = 0; i < prm->n_outer; ++i) {
    const double eta = eta_at(i, *prm, P.lambda);
    CS_CUDA(mark(p, TM_EULER, true), "event");
    cudaError_t e = launch_euler(P, S, *prm, i, eta, timeout_cycles);
    if (e != cudaSuccess)
      return fail(CS_ECUDA, std::string("euler launch: ") + cudaGetErrorString(e) + " at " + euler_last_call());
    if (prm->readout == CS_READOUT_BEST) {
      CS_CUDA(launch_readout(S.e_hist, S.s_hist, S.sigma, (int)P.N, S.trials, prm->n_steps, S.plan_ctas, P.stream),
              "readout launch");
      P.launches += 1;
    }
    CS_CUDA(mark(p, TM_EULER, false), "event");
    CS_CUDA(mark(p, TM_REFIT, true), "event");
    const RefitPlan rplan{prm->refit, prm->jacobi_iters, (int)P.N, P.num_sms, S.R};
    CS_CUDA(launch_refit(S.job, 1, S.trials, S.work, S.work_stride, S.work_blocks, i, P.stream, &rplan),
            "refit launch");
    if (refit_grid_wide(&rplan, 1, S.trials, S.work_blocks, S.work_stride)) P.launches += prm->jacobi_iters - 1;
    if (prm->record_outer) {
      const size_t nt = (size_t)P.N * S.trials;
      CS_CUDA(cudaMemcpyAsync(S.sig_outer + (size_t)i * nt, S.sigma, nt, cudaMemcpyDeviceToDevice, P.stream),
              "record outer support");
      CS_CUDA(cudaMemcpyAsync(S.R_outer + (size_t)i * nt, S.R, nt * sizeof(double), cudaMemcpyDeviceToDevice,
                              P.stream),
              "record outer signal");
    }
    CS_CUDA(mark(p, TM_REFIT, false), "event");
    P.launches += 2;
  }
  CS_CUDA(mark(p, TM_OTHER, true), "event");
  CS_CUDA(launch_finish(S.job, 1, S.trials, P.num_sms, P.stream, S.err4), "finish launch");
  CS_CUDA(mark(p, TM_OTHER, false), "event");
  P.launches += 4;  // energy, selection, error against FP64 and its ratio
  return CS_OK;
}

cs_status cs_solve(cs_problem* p, const cs_params* prm, int32_t trials) {
  if (!p) return fail(CS_EINVAL, "problem is NULL");
  cs_status st = check_params(prm, trials);
  if (st != CS_OK) return st;
  ProblemDev& P = p->P;
  SolveDev& S = p->S;
  S.done = false;
  p->n_marks = p->n_create_marks;
  P.launches = 2;
  CS_CUDA(mark(p, TM_OTHER, true), "event");
  if (P.gs_prec != prm->precision) ++P.launches;
  CS_CUDA(launch_store_coupling(P, prm->precision), "store coupling");
  if ((st = ensure_solve(P, S, *prm, trials)) != CS_OK) return st;
  CS_CUDA(clear_x(P, S), "memset X");
  CS_CUDA(cudaMemsetAsync(S.err, 0, sizeof(int), P.stream), "memset err");
  CS_CUDA(cudaMemsetAsync(S.singular, 0, sizeof(int), P.stream), "memset singular");
  int khz = 0;
  CS_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, P.device), "clock rate");
  const long long timeout_cycles = (long long)prm->timeout_ms * (long long)(khz > 0 ? khz : 2000000);
  const RefitJob hjob = make_job(P, S, *prm);
  CS_CUDA(cudaMemcpyAsync(S.job, &hjob, sizeof(hjob), cudaMemcpyHostToDevice, P.stream), "copy job");
  if (prm->init_R == CS_INIT_R_LASSO) {
    CS_CUDA(launch_lasso(P.G, P.hz, (int)P.N, S.trials, prm->lasso_lambda, prm->lasso_iters, S.work, S.R,
                         P.num_sms, P.stream),
            "LASSO initial R");
    P.launches += 2 * prm->lasso_iters + 2;
  } else {
    CS_CUDA(launch_init_R(S.job, 1, S.trials, P.num_sms, P.stream), "init R");
    P.launches += 1;
  }
  // the Euler plan of this shape (autotuning, if asked, times its candidates
  // here) and its streamed tiles, so that the loop below is stream work only
  {
    const cudaError_t e = launch_euler(P, S, *prm, 0, eta_at(0, *prm, P.lambda), timeout_cycles, true);
    if (e == cudaErrorInvalidConfiguration)
      return fail(CS_EINVAL, prm->tensor_form >= 2
                                 ? "tensor_form >= 2: no tensor-core work split of that kind for this shape and trials"
                                 : "N too large for the on-chip Euler kernel at this precision");
    if (e != cudaSuccess)
      return fail(CS_ECUDA, std::string("euler plan: ") + cudaGetErrorString(e) + " at " + euler_last_call());
  }
  CS_CUDA(mark(p, TM_OTHER, false), "event");
  const int64_t eager = P.launches - 2;  // kernels queued directly (coupling copy, initial R)
  // Every outer iteration and the objective are captured into one CUDA graph
  // and submitted to the problem's stream as a single launch (captured on a
  // private stream: the problem's stream may be the legacy default stream).
  reap_graphs();
  cudaStream_t user = P.stream, cap = nullptr;
  CS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "create the capture stream");
  {
    const cudaError_t eb = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (eb != cudaSuccess) {
      cudaStreamDestroy(cap);
      CS_CUDA(eb, "begin graph capture");
    }
  }
  P.stream = cap;
  p->capturing = true;
  st = queue_outer_loop(p, prm, timeout_cycles);
  p->capturing = false;
  P.stream = user;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
  cudaStreamDestroy(cap);
  if (st != CS_OK || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (st != CS_OK) return st;
    CS_CUDA(ec, "end graph capture");
  }
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CS_CUDA(e, "instantiate the solve graph");
  CS_CUDA(launch_and_keep(exec, user), "launch the solve graph");
  p->submissions = eager + 1;
  S.has_outer = prm->record_outer != 0;
  S.done = true;
  return CS_OK;
}

// Cluster size, span threshold and ring shape of a batched launch; the
// problems (row tiles in processing order, largest first) with at least
// span_rt row tiles are each run by a whole cluster.
static void apply_batch_shape(const BatchShape& sh, const std::vector<int>& rts, BatchLaunch* L) {
  L->cc = sh.cc;
  L->tps = sh.tps;
  L->slots = sh.slots;
  L->n_large = 0;
  if (sh.cc > 1)
    while (L->n_large < (int)rts.size() && rts[L->n_large] >= sh.span_rt) ++L->n_large;
}

// Batch autotuner: the shape of the group's launches (BatchShape), chosen
// by timing kBatchTuneSteps Euler steps of every problem of the group's first
// outer iteration for each candidate (clusters of 1, 2, 4, 8 CTAs, where a
// problem has at least two row tiles per CTA of a cluster, or only the
// cluster size the group's first problem fixes with cluster_size; 4, 2 or 1 column
// tiles per ring slot with as many slots as fit), twice each on the problems'
// stream (the second run counts), unless the tuning cache holds a choice for
// the group's precision, trials, form and row-tile histogram on this device.
// The runs write only the solves' scratch (state, X, sigma), which the real
// launches rewrite.
constexpr int kBatchTuneSteps = 48;

static cs_status tune_batch_shape(BatchLaunch L, const std::vector<int>& rts, int btc, int fixed_cc, int device,
                                  cudaStream_t stream, BatchShape* out) {
  std::map<int, int> hist;
  for (int r : rts) ++hist[r];
  std::string key = "batch|" + tune_device_tag(device) + "|p" + std::to_string(L.prm->precision) + "|T" +
                    std::to_string(L.T) + "|tc" + std::to_string(btc) + "|c" + std::to_string(L.ctas) + "|k" +
                    std::to_string(fixed_cc) + "|";
  for (const auto& kv : hist) key += std::to_string(kv.first) + ":" + std::to_string(kv.second) + ",";
  const int max_rt = rts.empty() ? 0 : *std::max_element(rts.begin(), rts.end());
  std::vector<BatchShape> cands;
  for (int cc : {1, 2, 4, 8}) {
    if ((cc > 1 && max_rt < 2 * cc && cc != fixed_cc) || (fixed_cc > 0 && cc != fixed_cc)) continue;
    for (int tps : {4, 2, 1}) {
      BatchShape b;
      b.cc = cc;
      b.tps = tps;
      b.slots = 0;
      b.span_rt = cc > 1 ? 2 * cc : 0;
      cands.push_back(b);
    }
  }
  auto tag = [](const BatchShape& b) {
    return std::to_string(b.cc) + " " + std::to_string(b.tps) + " " + std::to_string(b.slots) + " " +
           std::to_string(b.span_rt);
  };
  std::string stored;
  if (tune_lookup(key, &stored))
    for (const BatchShape& b : cands)
      if (tag(b) == stored) {
        *out = b;
        tune_note(false);
        return CS_OK;
      }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CS_CUDA(cudaEventCreate(&e0), "tuning event");
  cudaError_t e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    CS_CUDA(e, "tuning event");
  }
  float best = 0.f;
  bool have = false;
  L.step_cap = kBatchTuneSteps;
  for (const BatchShape& b : cands) {
    apply_batch_shape(b, rts, &L);
    float ms = 0.f;
    bool fits = true;
    for (int rep = 0; rep < 2 && e == cudaSuccess && fits; ++rep) {
      e = cudaEventRecord(e0, stream);
      if (e == cudaSuccess) {
        e = launch_euler_batch(L, stream);
        if (e == cudaErrorInvalidConfiguration) {  // the ring shape does not fit shared memory
          cudaGetLastError();
          e = cudaSuccess;
          fits = false;
        }
      }
      if (e == cudaSuccess && fits) e = cudaEventRecord(e1, stream);
      if (e == cudaSuccess && fits) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess && fits) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e != cudaSuccess) break;
    if (fits && (!have || ms < best)) {
      best = ms;
      *out = b;
      have = true;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CS_CUDA(e, "batch autotuning run");
  if (!have) return fail(CS_EINVAL, "batched Euler kernel does not fit shared memory");
  int err = 0;
  CS_CUDA(cudaMemcpy(&err, L.err, sizeof(int), cudaMemcpyDeviceToHost), "read tuning error word");
  if (err == DEV_TIMEOUT) return fail(CS_ETIMEOUT, "a device-side wait timed out while tuning the batch");
  tune_note(true);
  tune_store(key, tag(*out));
  return CS_OK;
}

cs_status cs_solve_batch(cs_problem* const* ps, const cs_params* const* prms, const int32_t* trials, int32_t n) {
  return cs::solve_batch(ps, prms, trials, n, nullptr);
}

}  // extern "C"

// cs_solve_batch with problem i drawing its initial amplitudes with instance
// number instances[i] (NULL: i).
cs_status cs::solve_batch(cs_problem* const* ps, const cs_params* const* prms, const int32_t* trials, int32_t n,
                          const int32_t* instances) {
  if (!ps || !prms || !trials || n < 1) return fail(CS_EINVAL, "need at least one problem, with its params and trials");
  for (int i = 0; i < n; ++i) {
    if (!ps[i]) return fail(CS_EINVAL, "problem is NULL");
    cs_status st = check_params(prms[i], trials[i]);
    if (st != CS_OK) return st;
    if (trials[i] > 64) return fail(CS_EINVAL, "a batched solve takes at most 64 trials per problem");
    if (prms[i]->record_steps != 0 || prms[i]->record_outer != 0)
      return fail(CS_EINVAL, "a batched solve does not record trajectories or outer histories");
    if (prms[i]->init_R != CS_INIT_R_ZEEMAN)
      return fail(CS_EINVAL, "a batched solve starts from R = h^z / diag G (init_R = CS_INIT_R_ZEEMAN)");
    if (prms[i]->readout != CS_READOUT_FINAL)
      return fail(CS_EINVAL, "a batched solve reads out the final configuration only (readout = CS_READOUT_FINAL)");
    if (ps[i]->P.stream != ps[0]->P.stream || ps[i]->P.device != ps[0]->P.device)
      return fail(CS_EINVAL, "the problems of a batch must share one stream and device");
    for (int k = 0; k < i; ++k)
      if (ps[k] == ps[i]) return fail(CS_EINVAL, "a problem appears twice in one batch");
  }
  ProblemDev& P0 = ps[0]->P;
  cudaStream_t stream = P0.stream;
  g_alloc_stream = stream;
  // Groups of problems that one batched launch can take: the same storage
  // precision, trial count and tensor-core decision.  Within a group the jobs
  // are ordered by n_outer (descending), so the problems still running at outer
  // iteration `it` are a prefix of the group.
  struct Group {
    int precision, T;
    int btc;  // batch_tc_kind
    std::vector<int> idx;
  };
  std::vector<Group> groups;
  std::vector<int> btcs(n);
  for (int i = 0; i < n; ++i) {
    const cs_params& p = *prms[i];
    const int btc = batch_tc_kind(p.precision, trials[i], p.tensor_form);
    if (p.tensor_form >= 2 && btc == 0)
      return fail(CS_EINVAL, "tensor_form >= 2: the batched tensor-core form needs BF16 or FP16 storage and 8 or 16 "
                             "trials");
    btcs[i] = btc;
    size_t g = 0;
    while (g < groups.size() &&
           !(groups[g].precision == p.precision && groups[g].T == trials[i] && groups[g].btc == btc))
      ++g;
    if (g == groups.size()) groups.push_back(Group{p.precision, trials[i], btc, {}});
    groups[g].idx.push_back(i);
  }
  int n_outer_max = 0;
  int64_t nmax = 0;
  int refit_items_max = 0;
  cs_status st = CS_OK;
  for (Group& G : groups) {
    // n_outer descending (the problems still running at iteration `it` are a
    // prefix), then N descending (the refit's work queue takes the large first)
    std::stable_sort(G.idx.begin(), G.idx.end(), [&](int a, int b) {
      return prms[a]->n_outer != prms[b]->n_outer ? prms[a]->n_outer > prms[b]->n_outer : ps[a]->P.N > ps[b]->P.N;
    });
    refit_items_max = std::max(refit_items_max, (int)G.idx.size() * G.T);
  }
  for (int i = 0; i < n; ++i) {
    ProblemDev& P = ps[i]->P;
    SolveDev& S = ps[i]->S;
    S.done = false;
    nmax = std::max(nmax, P.N);
    n_outer_max = std::max(n_outer_max, prms[i]->n_outer);
    CS_CUDA(launch_store_tiled(P, prms[i]->precision, btcs[i]), "store tiled coupling");
    if ((st = ensure_solve(P, S, *prms[i], trials[i], false)) != CS_OK) return st;
    CS_CUDA(clear_x(P, S), "memset X");
    CS_CUDA(cudaMemsetAsync(S.singular, 0, sizeof(int), stream), "memset singular");
  }
  // batch-owned buffers, released (stream-ordered) after the graph
  const size_t ib = batch_inst_bytes();
  // descriptors: for every outer iteration and group, the problems still running, largest N first
  std::vector<unsigned char> hinst;
  std::vector<std::vector<size_t>> inst_off(n_outer_max, std::vector<size_t>(groups.size(), 0));
  std::vector<std::vector<int>> inst_cnt(n_outer_max, std::vector<int>(groups.size(), 0));
  std::vector<std::vector<std::vector<int>>> inst_rt(n_outer_max, std::vector<std::vector<int>>(groups.size()));
  for (int it = 0; it < n_outer_max; ++it)
    for (size_t g = 0; g < groups.size(); ++g) {
      std::vector<int> act;
      for (int i : groups[g].idx)
        if (prms[i]->n_outer > it) act.push_back(i);
      std::stable_sort(act.begin(), act.end(), [&](int a, int b) { return ps[a]->P.N > ps[b]->P.N; });
      inst_off[it][g] = hinst.size();
      inst_cnt[it][g] = (int)act.size();
      for (int i : act) inst_rt[it][g].push_back(batch_row_tiles(ps[i]->P.N));
      hinst.resize(hinst.size() + ib * act.size());
      for (size_t k = 0; k < act.size(); ++k) {
        const int i = act[k];
        const double eta = eta_at(it, *prms[i], ps[i]->P.lambda);
        fill_batch_inst(hinst.data() + inst_off[it][g] + ib * k, ps[i]->P, ps[i]->S, *prms[i],
                        std::sqrt(prms[i]->tau) * eta * eta / 4.0, instances ? instances[i] : i);
      }
    }
  // refit jobs: per group, in the group's order (n_outer descending)
  std::vector<RefitJob> jobs;
  std::vector<size_t> job_off(groups.size());
  void* d_insts = nullptr;
  int* d_order = nullptr;
  int* d_queue = nullptr;
  int* d_err = nullptr;
  RefitJob* d_jobs = nullptr;
  double* pool = nullptr;
  double* d_err4 = nullptr;
  CS_CUDA(alloc(&d_err, 1), "cudaMalloc batch error word");
  for (size_t g = 0; g < groups.size(); ++g) {
    job_off[g] = jobs.size();
    for (int i : groups[g].idx) {
      jobs.push_back(make_job(ps[i]->P, ps[i]->S, *prms[i]));
      jobs.back().err = d_err;
    }
  }
  const size_t stride = (size_t)nmax * nmax + 4 * (size_t)nmax;
  int pool_blocks = std::min(refit_items_max, P0.num_sms);
  while (pool_blocks > 1 && (double)pool_blocks * stride * 8.0 > 16e9) --pool_blocks;
  CS_CUDA(dev_alloc(&d_insts, std::max<size_t>(hinst.size(), 1), stream), "cudaMalloc batch descriptors");
  CS_CUDA(alloc(&d_order, n), "cudaMalloc batch order");
  CS_CUDA(alloc(&d_queue, 1), "cudaMalloc batch queue");
  CS_CUDA(alloc(&d_jobs, n), "cudaMalloc batch jobs");
  CS_CUDA(alloc(&d_err4, 4 * (size_t)n), "cudaMalloc batch error scratch");
  CS_CUDA(alloc(&pool, (size_t)pool_blocks * stride), "cudaMalloc batch refit workspace");
  CS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), stream), "memset err");
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;  // descriptors are stored in processing order
  CS_CUDA(cudaMemcpyAsync(d_order, order.data(), n * sizeof(int), cudaMemcpyHostToDevice, stream), "copy order");
  CS_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), n * sizeof(RefitJob), cudaMemcpyHostToDevice, stream), "copy jobs");
  CS_CUDA(cudaMemcpyAsync(d_insts, hinst.data(), hinst.size(), cudaMemcpyHostToDevice, stream), "copy descriptors");
  int khz = 0;
  CS_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, P0.device), "clock rate");
  long long timeout_ms = 0;
  for (int i = 0; i < n; ++i) timeout_ms = std::max<long long>(timeout_ms, prms[i]->timeout_ms);
  const long long timeout_cycles = timeout_ms * (long long)(khz > 0 ? khz : 2000000);
  for (size_t g = 0; g < groups.size(); ++g)
    CS_CUDA(launch_init_R(d_jobs + job_off[g], (int)groups[g].idx.size(), groups[g].T, P0.num_sms, stream), "init R");
  // ring and cluster shape of each group: tuned (or taken from the tuning
  // cache) when a problem of the group asks for autotuning, else the default
  std::vector<BatchShape> shapes(groups.size());
  for (size_t g = 0; g < groups.size(); ++g) {
    bool tune = false;
    for (int i : groups[g].idx) tune = tune || prms[i]->autotune != 0;
    const int fixed_cc = prms[groups[g].idx[0]]->cluster_size;
    if (fixed_cc > 1) {
      shapes[g].cc = fixed_cc;
      shapes[g].span_rt = 2 * fixed_cc;
    }
    if (!tune || inst_cnt[0][g] == 0) continue;
    BatchLaunch L;
    L.insts = static_cast<unsigned char*>(d_insts) + inst_off[0][g];
    L.order = d_order;
    L.n = inst_cnt[0][g];
    L.T = groups[g].T;
    L.prm = prms[groups[g].idx[0]];
    L.queue = d_queue;
    L.outer = 0;
    L.err = d_err;
    L.timeout_cycles = timeout_cycles;
    L.ctas = L.prm->max_ctas > 0 ? std::min(L.prm->max_ctas, P0.num_sms) : P0.num_sms;
    if ((st = tune_batch_shape(L, inst_rt[0][g], groups[g].btc, fixed_cc, P0.device, stream, &shapes[g])) != CS_OK)
      return st;
  }
  CS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), stream), "memset err");
  // Every outer iteration of every group (batched Euler launch + refit) and the
  // objective are captured into one CUDA graph and submitted as a single launch.
  // (captured on a private stream: the problems' stream may be the legacy
  // default stream, which cannot be captured; the graph then runs on theirs)
  reap_graphs();
  cudaGraph_t graph = nullptr;
  cudaStream_t cap = nullptr;
  CS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "create the capture stream");
  {
    const cudaError_t eb = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (eb != cudaSuccess) {
      cudaStreamDestroy(cap);
      CS_CUDA(eb, "begin graph capture");
    }
  }
  cudaError_t e = cudaSuccess;
  const char* where = "";
  // phase timings of the whole batch, kept on the first problem (event-record
  // nodes of the graph; read with cs_problem_timing on ps[0])
  cs_problem* tp = ps[0];
  const cudaStream_t tp_stream = tp->P.stream;
  tp->n_marks = tp->n_create_marks;
  tp->P.stream = cap;
  tp->capturing = true;
  auto tmark = [&](int cat, bool begin) {
    if (e == cudaSuccess) e = mark(tp, cat, begin);
  };
  for (int it = 0; it < n_outer_max && e == cudaSuccess; ++it) {
    for (size_t g = 0; g < groups.size() && e == cudaSuccess; ++g) {
      const int na = inst_cnt[it][g];
      if (na == 0) continue;
      const cs_params& gp = *prms[groups[g].idx[0]];
      BatchLaunch L;
      L.insts = static_cast<unsigned char*>(d_insts) + inst_off[it][g];
      L.order = d_order;
      L.n = na;
      L.T = groups[g].T;
      L.prm = &gp;
      L.queue = d_queue;
      L.outer = it;
      L.err = d_err;
      L.timeout_cycles = timeout_cycles;
      L.ctas = gp.max_ctas > 0 ? std::min(gp.max_ctas, P0.num_sms) : P0.num_sms;
      L.test_skip = gp.test_phantom_ctas > 0 ? 1 : 0;
      apply_batch_shape(shapes[g], inst_rt[it][g], &L);
      tmark(TM_EULER, true);
      if (e == cudaSuccess) e = launch_euler_batch(L, cap);
      where = "batched euler launch";
      tmark(TM_EULER, false);
      tmark(TM_REFIT, true);
      if (e == cudaSuccess) {
        e = launch_refit(d_jobs + job_off[g], na, groups[g].T, pool, stride, pool_blocks, it, cap, nullptr, d_queue);
        where = "batched refit launch";
      }
      tmark(TM_REFIT, false);
    }
  }
  tmark(TM_OTHER, true);
  for (size_t g = 0; g < groups.size() && e == cudaSuccess; ++g) {
    e = launch_finish(d_jobs + job_off[g], (int)groups[g].idx.size(), groups[g].T, P0.num_sms, cap,
                      d_err4 + 4 * job_off[g]);
    where = "batched finish launch";
  }
  tmark(TM_OTHER, false);
  tp->capturing = false;
  tp->P.stream = tp_stream;
  const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (e == cudaErrorInvalidConfiguration) return fail(CS_EINVAL, "batched Euler kernel does not fit shared memory");
    return fail(CS_ECUDA, std::string(e != cudaSuccess ? where : "end graph capture") + ": " +
                              cudaGetErrorString(e != cudaSuccess ? e : ec));
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CS_CUDA(e, "instantiate the batch graph");
  CS_CUDA(launch_and_keep(exec, stream), "launch the batch graph");
  dev_free(d_insts, stream);
  dev_free(d_order, stream);
  dev_free(d_queue, stream);
  dev_free(d_err, stream);
  dev_free(d_jobs, stream);
  dev_free(pool, stream);
  dev_free(d_err4, stream);
  for (size_t g = 0; g < groups.size(); ++g)
    for (int i : groups[g].idx) {
      ps[i]->S.done = true;
      ps[i]->S.has_outer = false;
      ps[i]->S.plan_cluster =
          (shapes[g].cc > 1 && batch_row_tiles(ps[i]->P.N) >= shapes[g].span_rt) ? shapes[g].cc : 1;
      ps[i]->S.plan_ctas = std::min((int)groups[g].idx.size(), P0.num_sms);
      ps[i]->S.plan_form = groups[g].btc == 2 ? 6 : (groups[g].btc == 1 ? 4 : 3);
    }
  return CS_OK;
}

extern "C" {

static cs_status wait_and_check(cs_problem* p, double* stats_out) {
  if (!p) return fail(CS_EINVAL, "problem is NULL");
  if (!p->S.done) return fail(CS_ENOTREADY, "no solve queued on this problem");
  CS_CUDA(cudaStreamSynchronize(p->P.stream), "synchronize");
  double st[CS_STATS_LEN];
  CS_CUDA(cudaMemcpy(st, p->S.stats, CS_STATS_LEN * sizeof(double), cudaMemcpyDeviceToHost), "copy stats");
  st[8] = p->S.plan_cluster;
  st[9] = p->S.plan_ctas;
  st[10] = p->S.plan_form;
  if (stats_out) std::memcpy(stats_out, st, sizeof(st));
  const int err = (int)st[3];
  if (err == DEV_TIMEOUT) return fail(CS_ETIMEOUT, "a device-side wait timed out");
  if (err != 0) return fail(CS_ECUDA, "device error word " + std::to_string(err));
  return st[2] != 0.0 ? CS_ESINGULAR : CS_OK;
}

cs_status cs_result(cs_problem* p, double* x_hat, uint8_t* sigma_hat, double* energy, double* stats) {
  double st[CS_STATS_LEN];
  cs_status s = wait_and_check(p, st);
  if (s != CS_OK && s != CS_ESINGULAR) return s;
  const size_t N = (size_t)p->P.N;
  if (x_hat) CS_CUDA(cudaMemcpy(x_hat, p->S.x_hat, N * sizeof(double), cudaMemcpyDeviceToHost), "copy x_hat");
  if (sigma_hat) CS_CUDA(cudaMemcpy(sigma_hat, p->S.sigma_hat, N, cudaMemcpyDeviceToHost), "copy sigma_hat");
  if (energy) *energy = st[7];
  if (stats) std::memcpy(stats, st, sizeof(st));
  if (s == CS_ESINGULAR) set_last_error("a refit used the ridge");
  return s;
}

cs_status cs_result_trials(cs_problem* p, double* R, uint8_t* sigma, double* energy, int32_t* support_sizes) {
  cs_status s = wait_and_check(p, nullptr);
  if (s != CS_OK && s != CS_ESINGULAR) return s;
  const size_t N = (size_t)p->P.N, T = (size_t)p->S.trials;
  if (R) CS_CUDA(cudaMemcpy(R, p->S.R, N * T * sizeof(double), cudaMemcpyDeviceToHost), "copy R");
  if (sigma) CS_CUDA(cudaMemcpy(sigma, p->S.sigma, N * T, cudaMemcpyDeviceToHost), "copy sigma");
  if (energy) CS_CUDA(cudaMemcpy(energy, p->S.energy, T * sizeof(double), cudaMemcpyDeviceToHost), "copy energy");
  if (support_sizes)
    CS_CUDA(cudaMemcpy(support_sizes, p->S.ssize, (size_t)p->S.n_outer * T * sizeof(int32_t),
                       cudaMemcpyDeviceToHost),
            "copy support sizes");
  return s;
}

cs_status cs_trajectory(cs_problem* p, double* c, double* e) {
  cs_status s = wait_and_check(p, nullptr);
  if (s != CS_OK && s != CS_ESINGULAR) return s;
  const size_t n = (size_t)p->S.record_steps * p->P.N * p->S.trials;
  if (c) CS_CUDA(cudaMemcpy(c, p->S.rec_c, n * sizeof(double), cudaMemcpyDeviceToHost), "copy rec_c");
  if (e) CS_CUDA(cudaMemcpy(e, p->S.rec_e, n * sizeof(double), cudaMemcpyDeviceToHost), "copy rec_e");
  return s;
}

cs_status cs_outer_history(cs_problem* p, uint8_t* sigma, double* R) {
  cs_status s = wait_and_check(p, nullptr);
  if (s != CS_OK && s != CS_ESINGULAR) return s;
  if (!p->S.has_outer) return fail(CS_EINVAL, "the last solve did not record its outer iterations (record_outer)");
  const size_t n = (size_t)p->S.n_outer * p->P.N * p->S.trials;
  if (sigma) CS_CUDA(cudaMemcpy(sigma, p->S.sig_outer, n, cudaMemcpyDeviceToHost), "copy outer supports");
  if (R) CS_CUDA(cudaMemcpy(R, p->S.R_outer, n * sizeof(double), cudaMemcpyDeviceToHost), "copy outer signals");
  return s;
}

cs_status cs_problem_gram(cs_problem* p, double* G, double* hz, double* g) {
  if (!p) return fail(CS_EINVAL, "problem is NULL");
  CS_CUDA(cudaStreamSynchronize(p->P.stream), "synchronize");
  const size_t N = (size_t)p->P.N;
  if (G) CS_CUDA(cudaMemcpy(G, p->P.G, N * N * sizeof(double), cudaMemcpyDeviceToHost), "copy G");
  if (hz) CS_CUDA(cudaMemcpy(hz, p->P.hz, N * sizeof(double), cudaMemcpyDeviceToHost), "copy hz");
  if (g) CS_CUDA(cudaMemcpy(g, p->P.g, N * sizeof(double), cudaMemcpyDeviceToHost), "copy g");
  return CS_OK;
}

cs_status cs_problem_timing(cs_problem* p, double* ms, int64_t* launches) {
  if (!p) return fail(CS_EINVAL, "problem is NULL");
  CS_CUDA(cudaStreamSynchronize(p->P.stream), "synchronize");
  double acc[CS_TIMING_LEN] = {0, 0, 0, 0, 0};
  for (int k = 0; k < p->n_marks; ++k) {
    float t = 0.f;
    CS_CUDA(cudaEventElapsedTime(&t, p->events[2 * k], p->events[2 * k + 1]), "event time");
    acc[p->cats[k]] += t;
  }
  acc[4] = (double)p->submissions;
  if (ms) std::memcpy(ms, acc, sizeof(acc));
  if (launches) *launches = p->P.launches;
  return CS_OK;
}

cs_status cs_problem_shape(const cs_problem* p, int64_t* M, int64_t* N) {
  if (!p) return fail(CS_EINVAL, "problem is NULL");
  if (M) *M = p->P.M;
  if (N) *N = p->P.N;
  return CS_OK;
}

void cs_problem_destroy(cs_problem* p) {
  if (!p) return;
  cudaStream_t st = p->P.stream;
  free_solve(p->S, st);
  free_problem(p->P);
  cudaStreamSynchronize(st);
  for (cudaEvent_t ev : p->events) cudaEventDestroy(ev);
  delete p;
}

}  // extern "C"
