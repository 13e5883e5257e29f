// Continuous-batching request loop (host code; the GPU work is the solver's own
// kernels).  A small request gets a grid sized to its work (Euler CTAs, each a
// whole SM: about one per 26 million coupling FMAs per step and per 150 KB of
// G_off, at least 2) and runs as a cooperative launch with clusters of one CTA,
// so several small requests share the GPU with every grid resident.  A request
// whose grid would be more than half the GPU is large: it runs with the
// planner's own work split (clusters) over all SMs but a reserve of kBackfillSms
// (or the caller's cluster_size and max_ctas), one large request at a time, and
// the small requests admitted beside it run in the SMs it leaves.  A large
// request starts once no other large one runs and the small ones running fit in
// its reserve: a cluster launch does not keep its grid resident beside other
// grids, so a cluster that finds its SMs taken waits (bounded) until the small
// grid there ends; small grids never wait on the large one, so that costs time,
// not progress.  Requests are admitted whenever a slot (a CUDA stream of the
// server) is free, the request's device-memory estimate fits the remaining HBM
// budget and its grid fits the SMs not held by running requests; the queue is
// scanned in arrival order, a small request that does not fit yet does not hold
// back smaller ones behind it, and a large one at the head of the queue stops
// further admissions until it can start.
// Each admitted request forms its problem (or takes the caller's, whose G is
// already on the device) and queues its solve on its slot's stream, so the work
// of several requests overlaps on the GPU.  A worker thread harvests finished
// requests by event query, copies their results to host memory and frees their
// device memory, SMs and slot at once, which is what lets the next requests
// in.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3 };

struct Request {
  uint64_t ticket = 0;
  std::vector<double> A, y;
  int64_t M = 0, N = 0;
  double lambda = 0.0;
  cs_params prm;
  int trials = 0;
  size_t bytes = 0;
  bool alone = false;  // large: one at a time, small requests backfill the SMs it leaves
  int state = RQ_QUEUED;
  int slot = -1;
  cs_problem* p = nullptr;
  cs_problem* user = nullptr;       // the caller's problem (submitted by problem), else NULL
  cudaStream_t user_stream = nullptr;  // its own stream, restored when the request ends
  cudaEvent_t ev = nullptr;
  std::vector<double> x_hat;
  std::vector<uint8_t> sigma_hat;
  double energy = 0.0;
  double stats[CS_STATS_LEN] = {};
  cs_status status = CS_OK;
  std::string error;
  double t_submit = 0, t_start = 0, t_done = 0;
};

// Device bytes a request holds while it runs (problem, coupling copy, solve state,
// refit workspace), rounded up generously; without A and G when the problem is
// the caller's (already on the device).
size_t request_bytes(int64_t M, int64_t N, int trials, int precision, bool own_problem = true) {
  const size_t n = (size_t)N, m = (size_t)M, T = (size_t)trials;
  const size_t np = (n + cs::kPadN - 1) / cs::kPadN * cs::kPadN;
  const size_t gb = cs::storage_bytes(precision);
  const size_t cb = precision == CS_P_FP64 ? 8 : 4;
  size_t b = (own_problem ? m * n * 8 + n * n * 8 : 0) + np * np * gb;  // A, G, G_off
  b += n * T * (8 + 3 * cb + 1 + 4) + 2 * np * ((T + 3) / 4 * 4) * cb;  // R, state, sigma, sidx, X
  b += std::min<size_t>(T, 152) * (n * n + 2 * n) * 8;      // refit workspace
  return b + (1u << 20);
}

// Euler CTAs for a request: one per 26e6 coupling FMAs per step (N^2 T), and
// enough that each holds at most about 150 KB of G_off on chip, at least 2; at
// least kFp64MinCtas for FP64 problems, whose FMAs issue at a small fraction of
// the FP32 rate on this GPU (measured, N = 200 FP64: 27 us per step on 3 CTAs,
// 18 on 8).
constexpr int kFp64MinCtas = 8;

int server_grid(int num_sms, int64_t N, int trials, int precision) {
  const double work = (double)N * (double)N * (double)trials;
  const double gbytes = (double)N * (double)N * (double)cs::storage_bytes(precision);
  int d = (int)std::max(std::ceil(work / 26.0e6), std::ceil(gbytes / 150.0e3));
  if (precision == CS_P_FP64) d = std::max(d, kFp64MinCtas);
  return std::max(2, std::min(d, num_sms));
}

}  // namespace

struct cs_server {
  size_t budget = 0, in_use = 0;
  int max_slots = 0, device = 0, num_sms = 0, sms_in_use = 0;
  std::vector<cudaStream_t> streams;
  std::vector<char> slot_busy;
  std::deque<Request*> queue;
  std::vector<Request*> running;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::map<cs_problem*, int> busy;  // caller's problems with a request running (one at a time each)
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;

  int sms_of(const Request* r) const { return r->prm.max_ctas > 0 ? r->prm.max_ctas : num_sms; }

  void finish(Request* r) {
    r->status = cs_result(r->p, r->x_hat.data(), r->sigma_hat.data(), &r->energy, r->stats);
    if (r->status != CS_OK && r->status != CS_ESINGULAR) r->error = cs_last_error();
    release_problem(r);
    cudaEventDestroy(r->ev);
    r->ev = nullptr;
    r->state = (r->status == CS_OK || r->status == CS_ESINGULAR) ? RQ_DONE : RQ_FAILED;
    r->t_done = now_s();
    slot_busy[r->slot] = 0;
    in_use -= r->bytes;
    sms_in_use -= sms_of(r);
    r->A.clear();
    r->A.shrink_to_fit();
    r->y.clear();
    r->y.shrink_to_fit();
  }

  // The request's problem is done with: a problem the server formed is freed; a
  // caller's problem goes back to its own stream (its solve has completed, so
  // nothing is left on the server's stream) and is free for its next request.
  void release_problem(Request* r) {
    if (r->user) {
      cs::set_problem_stream(r->user, r->user_stream);
      busy.erase(r->user);
    } else if (r->p) {
      cs_problem_destroy(r->p);
    }
    r->p = nullptr;
  }

  // Admit r on slot s: form its problem (or take the caller's, moved onto the
  // slot's stream behind the work already queued on its own) and queue its solve
  // (caller holds mu).
  void start(Request* r, int s) {
    r->slot = s;
    slot_busy[s] = 1;
    in_use += r->bytes;
    sms_in_use += sms_of(r);
    r->t_start = now_s();
    r->x_hat.resize((size_t)r->N);
    r->sigma_hat.resize((size_t)r->N);
    cs_status st = CS_OK;
    if (r->user) {
      busy[r->user] = 1;
      r->p = r->user;
      r->user_stream = cs::problem_stream(r->user);
      cudaEvent_t before = nullptr;
      if (cudaEventCreateWithFlags(&before, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventRecord(before, r->user_stream) != cudaSuccess ||
          cudaStreamWaitEvent(streams[s], before, 0) != cudaSuccess) {
        cs::set_last_error("cannot order the request behind the problem's stream");
        st = CS_ECUDA;
      }
      if (before) cudaEventDestroy(before);
      if (st == CS_OK) cs::set_problem_stream(r->user, streams[s]);
    } else {
      st = cs_problem_create(r->A.data(), r->y.data(), r->M, r->N, r->lambda, 0, streams[s], &r->p);
    }
    if (st == CS_OK) st = cs_solve(r->p, &r->prm, r->trials);
    if (st == CS_OK && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) st = CS_ECUDA;
    if (st == CS_OK && cudaEventRecord(r->ev, streams[s]) != cudaSuccess) st = CS_ECUDA;
    if (st != CS_OK) {
      r->status = st;
      r->error = cs_last_error();
      if (r->user) cudaStreamSynchronize(streams[s]);
      release_problem(r);
      if (r->ev) cudaEventDestroy(r->ev);
      r->ev = nullptr;
      r->state = RQ_FAILED;
      r->t_done = now_s();
      slot_busy[s] = 0;
      in_use -= r->bytes;
      sms_in_use -= sms_of(r);
      return;
    }
    r->state = RQ_RUNNING;
    running.push_back(r);
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      bool progressed = false;
      for (size_t i = 0; i < running.size();) {
        Request* r = running[i];
        if (cudaEventQuery(r->ev) != cudaErrorNotReady) {
          finish(r);
          running.erase(running.begin() + i);
          progressed = true;
        } else {
          ++i;
        }
      }
      for (auto it = queue.begin(); it != queue.end();) {
        Request* r = *it;
        int s = -1;
        for (int i = 0; i < max_slots; ++i)
          if (!slot_busy[i]) { s = i; break; }
        if (s < 0) break;
        const bool held = r->user && busy.count(r->user);
        if (r->alone && !held) {
          bool large_running = false;
          for (const Request* q : running) large_running = large_running || q->alone;
          // wait (admitting nothing behind it) until it can start
          if (large_running || in_use + r->bytes > budget || sms_in_use + sms_of(r) > num_sms) break;
        }
        if (in_use + r->bytes > budget || sms_in_use + sms_of(r) > num_sms || held) {
          ++it;
          continue;
        }
        it = queue.erase(it);
        start(r, s);
        progressed = true;
      }
      if (progressed) cv.notify_all();
      if (running.empty() && queue.empty()) {
        cv.wait(lk, [&] { return stop || !queue.empty(); });
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
      }
    }
  }
};

extern "C" {

cs_status cs_server_create(size_t hbm_budget_bytes, int32_t max_slots, cs_server** out) {
  if (!out) {
    cs::set_last_error("out is NULL");
    return CS_EINVAL;
  }
  *out = nullptr;
  if (max_slots < 1 || max_slots > 256 || hbm_budget_bytes == 0) {
    cs::set_last_error("max_slots must be in [1, 256] and the budget positive");
    return CS_EINVAL;
  }
  cs_server* sv = new cs_server();
  sv->budget = hbm_budget_bytes;
  sv->max_slots = max_slots;
  if (cudaGetDevice(&sv->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, sv->device) != cudaSuccess) {
    cs::set_last_error("no CUDA device");
    delete sv;
    return CS_ECUDA;
  }
  sv->streams.resize(max_slots);
  sv->slot_busy.assign(max_slots, 0);
  for (int i = 0; i < max_slots; ++i) {
    if (cudaStreamCreateWithFlags(&sv->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaStreamDestroy(sv->streams[k]);
      cs::set_last_error("cudaStreamCreate failed");
      delete sv;
      return CS_ECUDA;
    }
  }
  sv->worker = std::thread([sv] { sv->loop(); });
  *out = sv;
  return CS_OK;
}

// SMs a large request leaves to the small requests that backfill beside it.
constexpr int kBackfillSms = 8;

// The server's share of the GPU for a request.  Small (a grid of at most half
// the SMs, sized to the work): cluster size 1 and cooperative launches, which
// keep every CTA of a grid resident while grids share SMs.  Large: one at a
// time, the caller's cluster_size and max_ctas (0: the planner's split over all
// SMs but kBackfillSms).
static bool server_params(const cs_server* sv, const cs_params* prm, int64_t N, int trials, cs_params* out) {
  *out = *prm;
  const int d = prm->max_ctas > 0 ? std::min(prm->max_ctas, sv->num_sms)
                                  : server_grid(sv->num_sms, N, trials, prm->precision);
  if (d > sv->num_sms / 2) {
    out->max_ctas = prm->max_ctas > 0 ? d : std::max(1, sv->num_sms - kBackfillSms);
    return true;
  }
  out->max_ctas = d;
  out->cluster_size = 1;
  return false;
}

static cs_status enqueue(cs_server* sv, std::unique_ptr<Request> r, uint64_t* ticket) {
  if (r->bytes > sv->budget) {
    cs::set_last_error("the request needs more device memory than the server's whole budget");
    return CS_ENOMEM;
  }
  r->t_submit = now_s();
  std::lock_guard<std::mutex> lk(sv->mu);
  r->ticket = sv->next_ticket++;
  *ticket = r->ticket;
  sv->queue.push_back(r.get());
  sv->reqs[r->ticket] = std::move(r);
  sv->cv.notify_all();
  return CS_OK;
}

cs_status cs_server_submit(cs_server* sv, cs_problem* p, const cs_params* prm, int32_t trials, uint64_t* ticket) {
  if (!sv || !p || !prm || !ticket) {
    cs::set_last_error("NULL argument");
    return CS_EINVAL;
  }
  if (trials < 1) {
    cs::set_last_error("trials must be >= 1");
    return CS_EINVAL;
  }
  std::unique_ptr<Request> r(new Request());
  r->user = p;
  r->M = cs::problem_M(p);
  r->N = cs::problem_N(p);
  r->alone = server_params(sv, prm, r->N, trials, &r->prm);
  r->trials = trials;
  r->bytes = request_bytes(r->M, r->N, trials, prm->precision, false);
  return enqueue(sv, std::move(r), ticket);
}

cs_status cs_server_submit_host(cs_server* sv, const double* A, const double* y, int64_t M, int64_t N, double lambda,
                                const cs_params* prm, int32_t trials, uint64_t* ticket) {
  if (!sv || !A || !y || !prm || !ticket) {
    cs::set_last_error("NULL argument");
    return CS_EINVAL;
  }
  if (M < 1 || N < 1 || trials < 1 || !(lambda >= 0.0)) {
    cs::set_last_error("bad sizes, trials or lambda");
    return CS_EINVAL;
  }
  std::unique_ptr<Request> r(new Request());
  r->M = M;
  r->N = N;
  r->lambda = lambda;
  r->alone = server_params(sv, prm, N, trials, &r->prm);
  r->trials = trials;
  r->bytes = request_bytes(M, N, trials, prm->precision);
  if (r->bytes <= sv->budget) {
    r->A.assign(A, A + (size_t)M * N);
    r->y.assign(y, y + (size_t)M);
  }
  return enqueue(sv, std::move(r), ticket);
}

cs_status cs_server_poll(cs_server* sv, uint64_t ticket, int32_t* done) {
  if (!sv || !done) {
    cs::set_last_error("NULL argument");
    return CS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) {
    cs::set_last_error("unknown ticket");
    return CS_EINVAL;
  }
  *done = it->second->state >= RQ_DONE ? 1 : 0;
  return CS_OK;
}

cs_status cs_server_wait(cs_server* sv, uint64_t ticket, int64_t timeout_ms) {
  if (!sv) {
    cs::set_last_error("NULL argument");
    return CS_EINVAL;
  }
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) {
    cs::set_last_error("unknown ticket");
    return CS_EINVAL;
  }
  Request* r = it->second.get();
  const bool ok = sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->state >= RQ_DONE; });
  if (!ok) {
    cs::set_last_error("request not finished within the timeout");
    return CS_ENOTREADY;
  }
  return CS_OK;
}

cs_status cs_server_result(cs_server* sv, uint64_t ticket, double* x_hat, uint8_t* sigma_hat, double* energy,
                           double* stats, double* times) {
  if (!sv) {
    cs::set_last_error("NULL argument");
    return CS_EINVAL;
  }
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
      cs::set_last_error("unknown ticket");
      return CS_EINVAL;
    }
    if (it->second->state < RQ_DONE) {
      cs::set_last_error("request not finished");
      return CS_ENOTREADY;
    }
    r = std::move(it->second);
    sv->reqs.erase(it);
  }
  if (r->state == RQ_FAILED) {
    cs::set_last_error(r->error);
    return r->status;
  }
  const size_t n = (size_t)r->N;
  if (x_hat) std::memcpy(x_hat, r->x_hat.data(), n * sizeof(double));
  if (sigma_hat) std::memcpy(sigma_hat, r->sigma_hat.data(), n);
  if (energy) *energy = r->energy;
  if (stats) std::memcpy(stats, r->stats, sizeof(r->stats));
  if (times) {
    times[0] = r->t_submit;
    times[1] = r->t_start;
    times[2] = r->t_done;
  }
  return r->status;
}

void cs_server_destroy(cs_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaSetDevice(sv->device);
  for (Request* r : sv->running) {
    cudaEventSynchronize(r->ev);
    sv->finish(r);
  }
  for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
  delete sv;
}

}  // extern "C"
