// Batch / serving executor: many homogenisation solves of different d, N, format and rank in flight on
// one GPU at once.  One solve leaves most of the GPU idle (its eigen-decompositions and Cholesky
// factors run one block per matrix, its products are small, and the host decides ranks and step
// lengths between launches), so throughput comes from overlapping independent solves: W worker
// threads, each with its own non-blocking CUDA stream and its own library context, take requests from
// a FIFO queue.  A request starts when a worker is free and its device footprint fits beside the
// footprints of the requests in flight within the executor's HBM budget (continuous batching:
// requests that arrive while others run are admitted as workers and memory free up).  The footprint of
// a request is the high-water mark of its context's pool measured on the last request of the same
// shape, or an estimate from its sizes before one has run.  Each request is a complete solve on its
// worker's context: its coefficient, cores and Krylov vectors stay on the device from upload to the
// A_eff evaluation, and its result does not depend on what else runs beside it.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <tuple>

#include "common.cuh"

using lrfg::DevicePool;

namespace {

using Clock = std::chrono::steady_clock;
// the quantities that fix a solve's memory use
using ShapeKey = std::tuple<int, int, int, int, int, int, int, int, int, int>;

struct Request {
  unsigned long long id = 0;
  lrfg_coeff coeff{};
  std::vector<double> parts[4];  // owned copies of the caller's host buffers
  double E[3] = {0, 0, 0};
  lrfg_opts opts{};
  ShapeKey key{};
  size_t footprint = 0;
  Clock::time_point submitted;
};

struct Done {
  bool ready = false;
  lrfg_status status = LRFG_OK;
  lrfg_result result{};
  lrfg_batch_report report{};
};

size_t grid_points(int d, const int* N) {
  size_t n = 1;
  for (int j = 0; j < d; ++j) n *= (size_t)N[j];
  return n;
}

int coeff_rank(const lrfg_coeff& c) {
  int r = 1;
  if (c.fmt == LRFG_TT)
    for (int j = 0; j <= c.d; ++j) r = std::max(r, c.tt.r[j]);
  if (c.fmt == LRFG_TUCKER || c.fmt == LRFG_CP)
    for (int j = 0; j < c.d; ++j) r = std::max(r, c.tk.r[j]);
  return r;
}

// device bytes a solve of this shape needs at its peak, before one has been measured
size_t estimate_footprint(const lrfg_coeff& c, const lrfg_opts& o) {
  const size_t n = grid_points(c.d, c.N);
  const size_t coeff_bytes = c.fmt == LRFG_FULL ? 8 * n : 0;
  if (o.fmt == LRFG_FULL) {
    // the coefficient, two real work grids and eight half-spectrum vectors
    const size_t half = n / c.N[c.d - 1] * ((c.N[c.d - 1] + 1) / 2);
    const size_t b = 8 * n * 3 + 16 * half * 8;
    if (o.disc == LRFG_GA) return b + (((size_t)24 * n) << c.d);  // double grid of about 2^d N^d points
    return o.prec == LRFG_MIXED ? b / 2 + 8 * n : b;
  }
  // low rank: the grid coefficient while it is compressed, and the Kronecker products of rank
  // s = r_A r that the operator forms (d components of N s^2 doubles, a few of them alive at once)
  size_t nmax = 0;
  for (int j = 0; j < c.d; ++j) nmax = std::max(nmax, (size_t)c.N[j]);
  const size_t s = (size_t)coeff_rank(c) * std::max(1, o.rank) * 2;
  return coeff_bytes * 2 + 8 * 8 * (size_t)c.d * nmax * s * s + (32u << 20);
}

}  // namespace

struct lrfg_batch {
  int device = 0;
  size_t budget = 0;
  size_t in_flight_bytes = 0;
  int running = 0;
  int pollers = 0;  // threads inside lrfg_batch_poll
  bool stopping = false;
  unsigned long long next_id = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Request>> queue;
  std::map<unsigned long long, Done> done;
  std::map<ShapeKey, size_t> measured;  // pool high-water mark of the last solve of each shape
  std::vector<size_t> reserved;         // bytes each worker's pool holds
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::vector<lrfg_ctx*> ctxs;
};

namespace {

size_t total(const std::vector<size_t>& v) {
  size_t s = 0;
  for (size_t x : v) s += x;
  return s;
}

void worker_loop(lrfg_batch* B, int w) {
  cudaSetDevice(B->device);
  lrfg_ctx* ctx = B->ctxs[w];
  DevicePool* pool = ctx->pool;
  for (;;) {
    std::unique_ptr<Request> req;
    {
      std::unique_lock<std::mutex> lock(B->mu);
      // FIFO admission: the head request starts when its footprint fits beside those in flight; a
      // request larger than the whole budget runs alone
      B->cv_work.wait(lock, [&] {
        if (B->stopping) return true;
        if (B->queue.empty()) return false;
        const size_t f = B->queue.front()->footprint;
        return B->running == 0 || B->budget == 0 || B->in_flight_bytes + f <= B->budget;
      });
      if (B->queue.empty()) {
        if (B->stopping) return;
        continue;
      }
      req = std::move(B->queue.front());
      B->queue.pop_front();
      auto m = B->measured.find(req->key);
      if (m != B->measured.end()) req->footprint = m->second;
      B->in_flight_bytes += req->footprint;
      ++B->running;
    }
    const Clock::time_point t0 = Clock::now();
    pool->reset_peak();
    const size_t base = pool->in_use();
    lrfg_result res{};
    const lrfg_status st = lrfg_solve(ctx, &req->coeff, req->E, &req->opts, &res, nullptr);
    const size_t peak = pool->peak() - base;
    const Clock::time_point t1 = Clock::now();
    bool trim = false;
    {
      std::lock_guard<std::mutex> lock(B->mu);
      B->in_flight_bytes -= req->footprint;
      --B->running;
      if (st == LRFG_OK || st == LRFG_ENOCONV) B->measured[req->key] = peak;
      B->reserved[w] = pool->reserved();
      trim = B->budget && total(B->reserved) > B->budget;
      Done& d = B->done[req->id];
      d.status = st;
      d.result = res;
      d.report.queue_s = std::chrono::duration<double>(t0 - req->submitted).count();
      d.report.run_s = std::chrono::duration<double>(t1 - t0).count();
      d.report.total_s = std::chrono::duration<double>(t1 - req->submitted).count();
      d.report.worker = w;
      d.report.peak_bytes = (double)peak;
      if (st != LRFG_OK) std::snprintf(d.report.message, sizeof(d.report.message), "%s", lrfg_last_error(ctx));
      d.ready = true;
    }
    if (trim) {
      // the pools together cache more than the budget: return this worker's cached blocks
      pool->trim();
      std::lock_guard<std::mutex> lock(B->mu);
      B->reserved[w] = pool->reserved();
    }
    B->cv_done.notify_all();
    B->cv_work.notify_all();
  }
}

lrfg_status copy_request(Request& req, const lrfg_coeff* c) {
  const int d = c->d;
  req.coeff = *c;
  if (c->fmt == LRFG_FULL) {
    if (!c->values) return LRFG_EINVAL;
    req.parts[0].assign(c->values, c->values + grid_points(d, c->N));
    req.coeff.values = req.parts[0].data();
  } else if (c->fmt == LRFG_TT) {
    if (c->tt.d != d) return LRFG_EINVAL;
    for (int j = 0; j < d; ++j) {
      if (!c->tt.cores[j] || c->tt.r[j] < 1 || c->tt.r[j + 1] < 1 || c->tt.N[j] < 1) return LRFG_EINVAL;
      const size_t n = (size_t)c->tt.r[j] * c->tt.N[j] * c->tt.r[j + 1];
      req.parts[j].assign(c->tt.cores[j], c->tt.cores[j] + n);
      req.coeff.tt.cores[j] = req.parts[j].data();
    }
  } else if (c->fmt == LRFG_TUCKER) {
    if (c->tk.d != d || !c->tk.core) return LRFG_EINVAL;
    size_t nc = 1;
    for (int j = 0; j < d; ++j) {
      if (c->tk.r[j] < 1 || c->tk.N[j] < 1 || !c->tk.factors[j]) return LRFG_EINVAL;
      nc *= (size_t)c->tk.r[j];
    }
    req.parts[3].assign(c->tk.core, c->tk.core + nc);
    req.coeff.tk.core = req.parts[3].data();
    for (int j = 0; j < d; ++j) {
      const size_t n = (size_t)c->tk.N[j] * c->tk.r[j];
      req.parts[j].assign(c->tk.factors[j], c->tk.factors[j] + n);
      req.coeff.tk.factors[j] = req.parts[j].data();
    }
  } else {
    return LRFG_EINVAL;
  }
  return LRFG_OK;
}

}  // namespace

extern "C" {

lrfg_status lrfg_batch_create(lrfg_batch** out, int device, int workers, size_t hbm_budget_bytes) {
  if (!out || workers < 1 || workers > 64) return LRFG_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return LRFG_ECUDA;
  }
  auto* B = new lrfg_batch();
  B->device = device;
  B->budget = hbm_budget_bytes;
  for (int w = 0; w < workers; ++w) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    lrfg_ctx* ctx = nullptr;
    // no cap on a worker's own pool (a request larger than the budget still runs, alone): admission
    // keeps the footprints in flight within the budget and trimming the cached blocks
    if (lrfg_create(&ctx, device, s, 0) != LRFG_OK) {
      cudaStreamDestroy(s);
      break;
    }
    B->streams.push_back(s);
    B->ctxs.push_back(ctx);
  }
  if ((int)B->ctxs.size() != workers) {
    for (size_t w = 0; w < B->ctxs.size(); ++w) {
      lrfg_destroy(B->ctxs[w]);
      cudaStreamDestroy(B->streams[w]);
    }
    delete B;
    return LRFG_ECUDA;
  }
  B->reserved.assign(workers, 0);
  for (int w = 0; w < workers; ++w) B->workers.emplace_back(worker_loop, B, w);
  *out = B;
  return LRFG_OK;
}

lrfg_status lrfg_batch_submit(lrfg_batch* B, const lrfg_coeff* coeff, const double* E, const lrfg_opts* opts,
                              unsigned long long* ticket) {
  if (!B || !coeff || !E || !opts || !ticket) return LRFG_EINVAL;
  if (coeff->on_device || coeff->d < 2 || coeff->d > 3) return LRFG_EINVAL;
  for (int j = 0; j < coeff->d; ++j)
    if (coeff->N[j] < 3 || coeff->N[j] % 2 == 0) return LRFG_EINVAL;
  auto req = std::make_unique<Request>();
  const lrfg_status st = copy_request(*req, coeff);
  if (st != LRFG_OK) return st;
  req->opts = *opts;
  for (int j = 0; j < coeff->d; ++j) req->E[j] = E[j];
  const int* N = coeff->N;
  req->key = ShapeKey(coeff->d, N[0], N[1], coeff->d == 3 ? N[2] : 1, (int)coeff->fmt, coeff_rank(*coeff),
                      (int)opts->fmt, (int)opts->prec, opts->rank, (int)opts->disc);
  req->footprint = estimate_footprint(*coeff, *opts);
  req->submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lock(B->mu);
    if (B->stopping) return LRFG_EINVAL;
    req->id = B->next_id++;
    *ticket = req->id;
    B->done[req->id] = Done{};
    B->queue.push_back(std::move(req));
  }
  B->cv_work.notify_all();
  return LRFG_OK;
}

lrfg_status lrfg_batch_poll(lrfg_batch* B, unsigned long long ticket, int wait, int* ready,
                            lrfg_status* solve_status, lrfg_result* res, lrfg_batch_report* report) {
  if (!B || !ready) return LRFG_EINVAL;
  std::unique_lock<std::mutex> lock(B->mu);
  if (B->done.find(ticket) == B->done.end()) return LRFG_EINVAL;
  ++B->pollers;
  if (wait) B->cv_done.wait(lock, [&] { return B->done[ticket].ready; });
  const Done d = B->done[ticket];
  *ready = d.ready ? 1 : 0;
  if (d.ready) {
    if (solve_status) *solve_status = d.status;
    if (res) *res = d.result;
    if (report) *report = d.report;
    B->done.erase(ticket);  // a completed result is handed out once
  }
  --B->pollers;
  B->cv_done.notify_all();  // lrfg_batch_destroy waits for the pollers to leave
  return LRFG_OK;
}

lrfg_status lrfg_batch_info(lrfg_batch* B, int* queued, int* running, size_t* in_flight_bytes) {
  if (!B) return LRFG_EINVAL;
  std::lock_guard<std::mutex> lock(B->mu);
  if (queued) *queued = (int)B->queue.size();
  if (running) *running = B->running;
  if (in_flight_bytes) *in_flight_bytes = B->in_flight_bytes;
  return LRFG_OK;
}

lrfg_status lrfg_batch_destroy(lrfg_batch* B) {
  if (!B) return LRFG_EINVAL;
  {
    std::lock_guard<std::mutex> lock(B->mu);
    B->stopping = true;
    // requests not yet started are dropped (a waiting poll returns them with LRFG_EINVAL); those running
    // finish first
    for (auto& r : B->queue) {
      Done& d = B->done[r->id];
      d.ready = true;
      d.status = LRFG_EINVAL;
      std::snprintf(d.report.message, sizeof(d.report.message), "%s",
                    "dropped: the executor was destroyed before the request started");
    }
    B->queue.clear();
  }
  B->cv_work.notify_all();
  B->cv_done.notify_all();
  for (auto& t : B->workers) t.join();
  {
    // no thread may still be inside lrfg_batch_poll when the executor is freed
    std::unique_lock<std::mutex> lock(B->mu);
    B->cv_done.wait(lock, [&] { return B->pollers == 0; });
  }
  cudaSetDevice(B->device);
  for (size_t w = 0; w < B->ctxs.size(); ++w) {
    lrfg_destroy(B->ctxs[w]);
    cudaStreamDestroy(B->streams[w]);
  }
  delete B;
  return LRFG_OK;
}

}  // extern "C"
