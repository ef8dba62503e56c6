// Serving loop: continuous batching of RPA energy requests on one GPU.
//
// Requests are deferred handles (inputs staged on the host).  A FIFO queue with backfill
// admits a request when a worker slot is free and its device-memory estimate fits in what is
// left of the server's HBM budget; a request at the head that has waited 2 s blocks backfill,
// so large requests are not starved.  Each slot is one host thread with one CUDA stream;
// allocations come from a stream-ordered memory pool (cudaMallocFromPoolAsync / cudaFreeAsync
// on the slot's stream), so freeing one request's memory does not synchronise the device and
// the admitted requests' kernels overlap.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace librpa {
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Ticket {
  librpa_gpu *h = nullptr;
  long long id = 0;
  int state = 0;   // 0 queued, 1 running, 2 done
  int rc = LIBRPA_OK;
  double ec = 0.0;
  Clock::time_point t_submit, t_admit, t_done;
  size_t est = 0, peak = 0;
  int slot = -1;
  bool exclusive = false;   // re-queued after a failed device allocation: runs alone
};

struct SlotCtx {
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
};

void *pool_alloc(size_t bytes, void *ctx) {
  SlotCtx *c = static_cast<SlotCtx *>(ctx);
  void *p = nullptr;
  if (cudaMallocFromPoolAsync(&p, bytes, c->pool, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void pool_free(void *p, void *ctx) { cudaFreeAsync(p, static_cast<SlotCtx *>(ctx)->stream); }

constexpr double kAgingMs = 2000.0;   // a head request waiting longer than this blocks backfill

}  // namespace
}  // namespace librpa

using namespace librpa;

struct librpa_gpu_server {
  int device = 0, nslots = 1;
  size_t budget = 0, in_use = 0, peak_reserved = 0;
  int running = 0, peak_running = 0;
  cudaMemPool_t pool = nullptr;
  std::vector<SlotCtx> slots;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<Ticket *> queue;
  std::map<long long, std::unique_ptr<Ticket>> tickets;
  std::map<librpa_gpu *, int> requests;   // handles made here -> 1 while submitted and unfinished
  long long next_id = 1, submitted = 0, completed = 0, failed = 0;
  std::vector<double> latency_ms;
  double queue_ms_sum = 0.0;
  bool any = false;
  Clock::time_point t_first, t_last;

  // under mu: the request to admit next, or nullptr
  Ticket *pick() {
    if (queue.empty()) return nullptr;
    const size_t avail = budget - in_use;
    Ticket *head = queue.front();
    if (head->exclusive) return running == 0 ? head : nullptr;   // no backfill past it
    if (head->est <= avail) return head;
    if (ms_between(head->t_submit, Clock::now()) > kAgingMs) return nullptr;
    for (Ticket *t : queue)
      if (t->est <= avail) return t;
    return nullptr;
  }

  void run(Ticket *t, int slot) {
    Handle &h = *t->h;
    const cudaStream_t own = h.stream;
    const librpa_gpu_opts saved = h.opts;
    h.stream = slots[slot].stream;
    h.opts.device = device;
    h.opts.dev_alloc = pool_alloc;
    h.opts.dev_free = pool_free;
    h.opts.alloc_ctx = &slots[slot];
    h.opts.hbm_budget = t->est;   // a wrong estimate fails this request, not its neighbours
    h.bytes_peak = 0;
    double ec = 0.0;
    int rc = librpa_gpu_chi0(t->h, nullptr, nullptr);
    if (rc == LIBRPA_OK) rc = librpa_gpu_ec(t->h, &ec, nullptr, nullptr);
    t->rc = rc;
    t->ec = ec;
    t->peak = h.bytes_peak;
    try {
      release_device(h);
    } catch (...) {
    }
    cudaStreamSynchronize(h.stream);
    h.stream = own;
    h.opts = saved;
  }

  void worker(int slot) {
    cudaSetDevice(device);
    for (;;) {
      Ticket *t = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || (t = pick()) != nullptr; });
        if (stop) return;
        queue.erase(std::find(queue.begin(), queue.end(), t));
        t->state = 1;
        t->slot = slot;
        t->t_admit = Clock::now();
        in_use += t->est;
        peak_reserved = std::max(peak_reserved, in_use);
        peak_running = std::max(peak_running, ++running);
      }
      run(t, slot);
      {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= t->est;
        --running;
        if (t->rc == LIBRPA_E_NOMEM && !t->exclusive && !stop) {
          // the device ran out although the estimates fit the budget (memory held outside the
          // server, pool fragmentation): run it again once, alone, at the head of the queue
          t->exclusive = true;
          t->state = 0;
          t->slot = -1;
          queue.push_front(t);
          cv.notify_all();
          continue;
        }
        t->t_done = Clock::now();
        t->state = 2;
        requests[t->h] = 0;
        if (t->rc == LIBRPA_OK) {
          ++completed;
          latency_ms.push_back(ms_between(t->t_submit, t->t_done));
          queue_ms_sum += ms_between(t->t_submit, t->t_admit);
          t_last = t->t_done;
        } else {
          ++failed;
        }
      }
      cv.notify_all();
    }
  }
};

extern "C" {

int librpa_gpu_estimate_bytes(librpa_gpu_t h, size_t *bytes) {
  if (!h || !bytes) return LIBRPA_E_ARG;
  if (!h->have_structure) {
    h->last_error = "estimate_bytes before set_structure";
    return LIBRPA_E_STATE;
  }
  try {
    *bytes = estimate_device_bytes(*h);
  } catch (const Error &e) {
    h->last_error = e.msg;
    return e.code;
  } catch (...) {
    h->last_error = "estimate_bytes: host failure";
    return LIBRPA_E_NOMEM;
  }
  return LIBRPA_OK;
}

int librpa_gpu_server_create(librpa_gpu_server_t *sp, const librpa_gpu_server_opts *o) {
  if (!sp || !o || o->slots < 1 || o->slots > 64) return LIBRPA_E_ARG;
  *sp = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return LIBRPA_E_CUDA;
  }
  if (o->device < 0 || o->device >= ndev) return LIBRPA_E_ARG;
  if (cudaSetDevice(o->device) != cudaSuccess) return LIBRPA_E_CUDA;
  std::unique_ptr<librpa_gpu_server> s(new (std::nothrow) librpa_gpu_server());
  if (!s) return LIBRPA_E_NOMEM;
  s->device = o->device;
  s->nslots = o->slots;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return LIBRPA_E_CUDA;
  s->budget = o->hbm_budget ? o->hbm_budget : (size_t)(0.9 * (double)fr);
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = o->device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) return LIBRPA_E_CUDA;
  uint64_t keep = UINT64_MAX;   // keep freed blocks in the pool for the next request
  cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  s->slots.resize(o->slots);
  for (SlotCtx &c : s->slots) {
    c.pool = s->pool;
    if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (SlotCtx &d : s->slots)
        if (d.stream) cudaStreamDestroy(d.stream);
      cudaMemPoolDestroy(s->pool);
      return LIBRPA_E_CUDA;
    }
  }
  librpa_gpu_server *raw = s.get();
  for (int i = 0; i < o->slots; ++i) raw->workers.emplace_back([raw, i] { raw->worker(i); });
  *sp = s.release();
  return LIBRPA_OK;
}

int librpa_gpu_server_request(librpa_gpu_server_t s, const librpa_gpu_opts *o, librpa_gpu_t *req) {
  if (!s || !o || !req) return LIBRPA_E_ARG;
  librpa_gpu_opts c = *o;
  c.device = s->device;
  c.stream = nullptr;
  c.dev_alloc = nullptr;
  c.dev_free = nullptr;
  c.alloc_ctx = nullptr;
  int rc = librpa_gpu_create(req, &c);
  if (rc != LIBRPA_OK) return rc;
  (*req)->deferred = true;
  std::lock_guard<std::mutex> lk(s->mu);
  s->requests[*req] = 0;
  return LIBRPA_OK;
}

int librpa_gpu_server_submit(librpa_gpu_server_t s, librpa_gpu_t req, long long *ticket) {
  if (!s || !req || !ticket) return LIBRPA_E_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->requests.find(req);
    if (it == s->requests.end()) return LIBRPA_E_ARG;
    if (it->second) {
      req->last_error = "server_submit: the request is already queued or running";
      return LIBRPA_E_STATE;
    }
  }
  req->last_error.clear();
  if (!req->have_structure) {
    req->last_error = "server_submit: set_structure missing";
    return LIBRPA_E_STATE;
  }
  for (int k = 0; k < req->mesh.size(); ++k)
    if (!req->have_k[k] || !req->have_q[k]) {
      req->last_error = "server_submit: set_green or set_coulomb missing for k/q index " + std::to_string(k);
      return LIBRPA_E_STATE;
    }
  size_t est = 0;
  int rc = librpa_gpu_estimate_bytes(req, &est);
  if (rc != LIBRPA_OK) return rc;
  std::unique_ptr<Ticket> t(new Ticket());
  t->h = req;
  t->est = est;
  t->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (est > s->budget) {
      req->last_error = "server_submit: the request needs about " + std::to_string(est) +
                        " device bytes, more than the server's budget of " + std::to_string(s->budget);
      return LIBRPA_E_NOMEM;
    }
    t->id = s->next_id++;
    *ticket = t->id;
    if (!s->any) {
      s->any = true;
      s->t_first = t->t_submit;
    }
    ++s->submitted;
    s->requests[req] = 1;
    s->queue.push_back(t.get());
    s->tickets[t->id] = std::move(t);
  }
  s->cv.notify_all();
  return LIBRPA_OK;
}

int librpa_gpu_server_wait(librpa_gpu_server_t s, long long ticket, double timeout_s, librpa_gpu_result *r) {
  if (!s || !r) return LIBRPA_E_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return LIBRPA_E_ARG;
  Ticket *t = it->second.get();
  auto done = [&] { return t->state == 2; };
  if (timeout_s < 0)
    s->cv.wait(lk, done);
  else if (!s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), done))
    return LIBRPA_E_TIMEOUT;
  r->status = t->rc;
  r->ec = t->ec;
  r->ms_queue = t->slot >= 0 ? ms_between(t->t_submit, t->t_admit) : ms_between(t->t_submit, t->t_done);
  r->ms_run = t->slot >= 0 ? ms_between(t->t_admit, t->t_done) : 0.0;
  r->ms_total = ms_between(t->t_submit, t->t_done);
  r->bytes_reserved = t->est;
  r->bytes_peak = t->peak;
  r->slot = t->slot;
  return LIBRPA_OK;
}

int librpa_gpu_server_get_stats(librpa_gpu_server_t s, librpa_gpu_server_stats *st) {
  if (!s || !st) return LIBRPA_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = librpa_gpu_server_stats{};
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  std::vector<double> l = s->latency_ms;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) {   // nearest rank
    if (l.empty()) return 0.0;
    size_t k = (size_t)std::ceil(p / 100.0 * (double)l.size());
    return l[std::min(l.size(), std::max<size_t>(k, 1)) - 1];
  };
  st->p50_ms = pct(50);
  st->p99_ms = pct(99);
  st->mean_queue_ms = s->completed ? s->queue_ms_sum / (double)s->completed : 0.0;
  const double span = s->completed ? ms_between(s->t_first, s->t_last) : 0.0;
  st->energies_per_s = span > 0 ? 1e3 * (double)s->completed / span : 0.0;
  st->peak_running = s->peak_running;
  st->peak_reserved = s->peak_reserved;
  st->hbm_budget = s->budget;
  return LIBRPA_OK;
}

void librpa_gpu_server_destroy(librpa_gpu_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Ticket *t : s->queue) {   // never admitted
      t->rc = LIBRPA_E_STATE;
      t->t_done = Clock::now();
      t->state = 2;
      s->requests[t->h] = 0;
    }
    s->queue.clear();
  }
  s->cv.notify_all();
  for (std::thread &w : s->workers) w.join();
  cudaSetDevice(s->device);
  for (SlotCtx &c : s->slots) {
    cudaStreamSynchronize(c.stream);
    cudaStreamDestroy(c.stream);
  }
  cudaMemPoolDestroy(s->pool);
  delete s;
}

}  // extern "C"
