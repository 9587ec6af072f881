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
#include <string>
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
  std::string group_key;  // requests with equal non-empty keys may be solved together in lockstep
  size_t footprint = 0;
  Clock::time_point submitted;
};

// The key of the requests that one lockstep solve (lrfg_problems_solve) can take together: isotropic GaNi TT
// solves at a fixed rank or with rank adaptation, of TT coefficients of equal grid and ranks, with equal options.
// Empty for every other request.
std::string lockstep_key(const lrfg_coeff& c, const lrfg_opts& o) {
  if (c.fmt != LRFG_TT || o.fmt != LRFG_TT || o.disc != LRFG_GANI || o.rank_tol != 0.0) return std::string();
  for (double b : c.B)
    if (b != 0.0) return std::string();
  char k[512];
  std::snprintf(k, sizeof(k), "%d|%d,%d,%d|%d,%d,%d,%d|%d|%d|%.17g|%.17g|%d|%d|%d|%d|%d|%u|%d", c.d, c.N[0], c.N[1],
                c.d == 3 ? c.N[2] : 1, c.tt.r[0], c.tt.r[1], c.tt.r[2], c.d == 3 ? c.tt.r[3] : 1, (int)o.prec, o.rank,
                o.pinv_eps, o.tol, o.maxit, o.stop_on_increase, o.rank_start, o.rank_step, o.sketch_over,
                o.sketch_seed, o.sketch_keep);
  return std::string(k);
}

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
  int group_max = 1;                    // requests of one lockstep key a worker takes together (1: one at a time)
  std::map<ShapeKey, size_t> measured;  // pool high-water mark per request of the last solve of each shape
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

// one request's status from its result, as lrfg_problem_solve gives it
lrfg_status member_status(const lrfg_result& r, const lrfg_opts& o) {
  const bool stopped = o.stop_on_increase && r.applies > 0 && r.iters < o.maxit;
  return (r.converged || stopped) ? LRFG_OK : LRFG_ENOCONV;
}

// Solve the requests of one group on the worker's context: one request by lrfg_solve; several (of one lockstep
// key) by lrfg_problems_solve over their problems, in lockstep.  st[i] / res[i] / msg[i] per request.
void run_group(lrfg_ctx* ctx, std::vector<std::unique_ptr<Request>>& g, std::vector<lrfg_status>& st,
               std::vector<lrfg_result>& res, std::vector<std::string>& msg) {
  const size_t n = g.size();
  st.assign(n, LRFG_OK);
  res.assign(n, lrfg_result{});
  msg.assign(n, std::string());
  if (n == 1) {
    st[0] = lrfg_solve(ctx, &g[0]->coeff, g[0]->E, &g[0]->opts, &res[0], nullptr);
    if (st[0] != LRFG_OK) msg[0] = lrfg_last_error(ctx);
    return;
  }
  std::vector<lrfg_problem*> ps;
  std::vector<size_t> who;
  std::vector<double> Es;
  for (size_t i = 0; i < n; ++i) {
    lrfg_problem* P = nullptr;
    st[i] = lrfg_problem_create(ctx, &g[i]->coeff, &g[i]->opts, &P);
    if (st[i] != LRFG_OK) {
      msg[i] = lrfg_last_error(ctx);
      continue;
    }
    ps.push_back(P);
    who.push_back(i);
    for (int j = 0; j < g[i]->coeff.d; ++j) Es.push_back(g[i]->E[j]);
  }
  if (!ps.empty()) {
    std::vector<lrfg_result> rs(ps.size());
    const lrfg_status s1 = lrfg_problems_solve((int)ps.size(), ps.data(), Es.data(), rs.data());
    const std::string m1 = s1 == LRFG_OK ? std::string() : std::string(lrfg_last_error(ctx));
    for (size_t k = 0; k < ps.size(); ++k) {
      const size_t i = who[k];
      res[i] = rs[k];
      st[i] = (s1 == LRFG_OK || s1 == LRFG_ENOCONV) ? member_status(rs[k], g[i]->opts) : s1;
      if (st[i] == LRFG_ENOCONV) msg[i] = lrfg_strerror(LRFG_ENOCONV);
      else if (st[i] != LRFG_OK) msg[i] = m1;
      lrfg_problem_free(ps[k]);
    }
  }
}

void worker_loop(lrfg_batch* B, int w) {
  cudaSetDevice(B->device);
  lrfg_ctx* ctx = B->ctxs[w];
  DevicePool* pool = ctx->pool;
  for (;;) {
    std::vector<std::unique_ptr<Request>> g;
    size_t footprint = 0;
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
      auto fp = [&](Request& r) {
        auto m = B->measured.find(r.key);
        if (m != B->measured.end()) r.footprint = m->second;
        return r.footprint;
      };
      g.push_back(std::move(B->queue.front()));
      B->queue.pop_front();
      footprint = fp(*g[0]);
      // continuous batching across requests: queued requests of the head's lockstep key join it (in queue
      // order, while their footprints fit), so that one launch sequence serves all of them
      const std::string key = g[0]->group_key;
      if (B->group_max > 1 && !key.empty()) {
        for (auto it = B->queue.begin(); it != B->queue.end() && (int)g.size() < B->group_max;) {
          if ((*it)->group_key == key) {
            const size_t f = fp(**it);
            if (B->budget == 0 || B->in_flight_bytes + footprint + f <= B->budget || B->running == 0) {
              footprint += f;
              g.push_back(std::move(*it));
              it = B->queue.erase(it);
              continue;
            }
          }
          ++it;
        }
      }
      B->in_flight_bytes += footprint;
      ++B->running;
    }
    const Clock::time_point t0 = Clock::now();
    pool->reset_peak();
    const size_t base = pool->in_use();
    std::vector<lrfg_status> st;
    std::vector<lrfg_result> res;
    std::vector<std::string> msg;
    run_group(ctx, g, st, res, msg);
    const size_t peak = pool->peak() - base;
    const Clock::time_point t1 = Clock::now();
    bool trim = false;
    {
      std::lock_guard<std::mutex> lock(B->mu);
      B->in_flight_bytes -= footprint;
      --B->running;
      bool ok = true;
      for (lrfg_status s1 : st) ok = ok && (s1 == LRFG_OK || s1 == LRFG_ENOCONV);
      // per request: a group's high-water mark shared out over its members
      if (ok) B->measured[g[0]->key] = (peak + g.size() - 1) / g.size();
      B->reserved[w] = pool->reserved();
      trim = B->budget && total(B->reserved) > B->budget;
      for (size_t i = 0; i < g.size(); ++i) {
        Done& d = B->done[g[i]->id];
        d.status = st[i];
        d.result = res[i];
        d.report.queue_s = std::chrono::duration<double>(t0 - g[i]->submitted).count();
        d.report.run_s = std::chrono::duration<double>(t1 - t0).count();
        d.report.total_s = std::chrono::duration<double>(t1 - g[i]->submitted).count();
        d.report.worker = w;
        d.report.group = (int)g.size();
        d.report.peak_bytes = (double)peak;
        if (st[i] != LRFG_OK) std::snprintf(d.report.message, sizeof(d.report.message), "%s", msg[i].c_str());
        d.ready = true;
      }
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
  req->group_key = lockstep_key(*coeff, *opts);
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

lrfg_status lrfg_batch_set_group(lrfg_batch* B, int max_requests) {
  if (!B || max_requests < 1 || max_requests > 32) return LRFG_EINVAL;
  std::lock_guard<std::mutex> lock(B->mu);
  B->group_max = max_requests;
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
