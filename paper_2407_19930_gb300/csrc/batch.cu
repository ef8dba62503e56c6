// Batched energies: many independent structures (handles) in one pass.  The FP64 chi0
// contraction of all single-channel FP64 handles runs in rounds of point batches on one stream,
// each round's GEMMs as single grouped launches over all those handles' tiles (uneven block
// shapes), with tile variants tuned on the first run and the launch sequence replayed from a
// CUDA graph afterwards.  The single-channel tensor-core handles are grouped by digit-plane count,
// and each group's chi0 contraction runs in rounds whose N-step, X-step and final GEMMs are one
// launch over all the group's tiles (tensor maps per handle).  Those groups and the remaining
// handles (nspins = 2, screening) run at the same time on up to four worker threads, each with
// its own stream, so that small structures overlap on the device.  G, the transforms and the ln
// det stage run per handle.
#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

using namespace librpa;

struct librpa_gpu_batch {
  std::vector<librpa_gpu *> hs;
  MergedChi0 m;
  librpa_gpu_batch_stats st{};
};

namespace {

struct StreamSwap {   // the merged handles on the first one's stream for the duration of a run
  std::vector<librpa_gpu *> &hs;
  std::vector<cudaStream_t> saved;
  explicit StreamSwap(std::vector<librpa_gpu *> &h) : hs(h) {
    for (librpa_gpu *x : hs) {
      saved.push_back(x->stream);
      x->stream = hs[0]->stream;
    }
  }
  ~StreamSwap() {
    for (size_t i = 0; i < hs.size(); ++i) hs[i]->stream = saved[i];
  }
};

struct Failure {
  int index = -1, code = LIBRPA_OK;
  std::string msg;
};

// The whole path of one handle on stream `ws` (G, plan, chi0, transforms, ln det), releasing its
// chi0(q, i omega) and workspace afterwards; throws Error.
void run_own(Handle &h, cudaStream_t ws, double *ec) {
  const cudaStream_t saved = h.stream;
  h.stream = ws;
  struct Restore {
    Handle &h;
    cudaStream_t s;
    ~Restore() { h.stream = s; }
  } restore{h, saved};
  materialize(h);
  h.stats = librpa_gpu_stats{};
  const double imag = green_build(h);
  if (h.lri_dirty) {
    chi0_plan(h);
    h.lri_dirty = false;
  }
  chi0_run(h, nullptr);
  freq_transform(h);
  h.chi0_done = true;
  const int rc = ec_run(h, ec, nullptr, nullptr);
  if (rc == LIBRPA_E_NOT_PD) throw Error{rc, "ec: a Cholesky pivot was <= 0"};
  if (rc) throw Error{rc, "ec: a bounded device wait ran out"};
  h.release(h.d_chi_qw);
  h.release(h.work);
  h.chi0_done = false;
  h.resolve_timers();
  if (h.opts.check_level >= 1 && !(imag <= 1e-10)) throw Error{LIBRPA_E_NUMERIC, "batch: G(R, tau) has an imaginary part"};
}

// A group of tensor-core handles with the same digit-plane count on stream `ws`: G per handle, the
// chi0 contraction of all of them merged (chi0_run_tc_merged), then transforms and ln det per
// handle, releasing each one's chi0(q, i omega) and workspace afterwards; throws Error with
// *failed set to the position in `g` of the handle concerned.
void run_tc_group(std::vector<Handle *> &g, cudaStream_t ws, double *const *ec, int *failed) {
  std::vector<cudaStream_t> saved;
  for (Handle *h : g) {
    saved.push_back(h->stream);
    h->stream = ws;
  }
  struct Restore {
    std::vector<Handle *> &g;
    std::vector<cudaStream_t> &s;
    ~Restore() {
      for (size_t i = 0; i < g.size(); ++i) g[i]->stream = s[i];
    }
  } restore{g, saved};
  std::vector<double> imag(g.size());
  for (size_t i = 0; i < g.size(); ++i) {
    *failed = (int)i;
    Handle &h = *g[i];
    materialize(h);
    h.stats = librpa_gpu_stats{};
    imag[i] = green_build(h);
    if (h.lri_dirty) {
      chi0_plan(h);
      h.lri_dirty = false;
    }
  }
  *failed = 0;
  chi0_run_tc_merged(g);
  for (size_t i = 0; i < g.size(); ++i) {
    *failed = (int)i;
    Handle &h = *g[i];
    freq_transform(h);
    h.chi0_done = true;
    const int rc = ec_run(h, ec[i], nullptr, nullptr);
    if (rc == LIBRPA_E_NOT_PD) throw Error{rc, "ec: a Cholesky pivot was <= 0"};
    if (rc) throw Error{rc, "ec: a bounded device wait ran out"};
    h.release(h.d_chi_qw);
    h.release(h.work);
    h.chi0_done = false;
    h.resolve_timers();
    if (h.opts.check_level >= 1 && !(imag[i] <= 1e-10)) throw Error{LIBRPA_E_NUMERIC, "batch: G(R, tau) has an imaginary part"};
  }
}

}  // namespace

extern "C" {

int librpa_gpu_batch_create(librpa_gpu_batch_t *bp, librpa_gpu_t *hs, int n) {
  if (!bp || !hs || n < 1) return LIBRPA_E_ARG;
  *bp = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return LIBRPA_E_ARG;
    if (hs[i]->opts.device != hs[0]->opts.device) return LIBRPA_E_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return LIBRPA_E_ARG;
  }
  librpa_gpu_batch *b = new (std::nothrow) librpa_gpu_batch();
  if (!b) return LIBRPA_E_NOMEM;
  b->hs.assign(hs, hs + n);
  b->st.n = n;
  b->st.var_nx = b->st.var_fin = -1;
  b->st.failed_index = -1;
  *bp = b;
  return LIBRPA_OK;
}

int librpa_gpu_batch_run(librpa_gpu_batch_t b, double *ec) {
  if (!b || !ec) return LIBRPA_E_ARG;
  std::vector<librpa_gpu *> &hs = b->hs;
  const int n = (int)hs.size();
  b->st.failed_index = -1;
  auto fail_at = [&](int i, int code, const std::string &msg) {
    hs[i]->last_error = msg;
    b->st.failed_index = i;
    return code;
  };
  const int dev = hs[0]->opts.device;
  cudaSetDevice(dev);
  for (int i = 0; i < n; ++i) {
    hs[i]->last_error.clear();
    if (int rc = chi0_prepare(*hs[i])) return fail_at(i, rc, hs[i]->last_error);
  }
  const auto t_start = std::chrono::steady_clock::now();
  std::vector<int> mi, oi;   // merged FP64 handles, handles on their own path
  std::map<int, std::vector<int>> tcg;   // tensor-core handles by digit-plane count (merged per group)
  for (int i = 0; i < n; ++i) {
    if (chi0_fits_one_batch(*hs[i]))
      mi.push_back(i);
    else if (chi0_fits_tc_batch(*hs[i]))
      tcg[hs[i]->chi0_S].push_back(i);
    else
      oi.push_back(i);
  }
  // worker jobs: a tensor-core group (one merged contraction) or one own-path handle
  std::vector<std::vector<int>> jobs;
  int n_tc_merged = 0;
  for (auto &kv : tcg) {
    jobs.push_back(kv.second);
    if (kv.second.size() > 1) n_tc_merged += (int)kv.second.size();
  }
  for (int i : oi) jobs.push_back({i});
  // up to four workers, each on its own stream
  std::mutex fmu;
  Failure own_fail;
  long long own_launches = 0;
  const int nwk = std::min<int>(4, (int)jobs.size());
  std::vector<std::thread> workers;
  for (int w = 0; w < nwk; ++w)
    workers.emplace_back([&, w] {
      cudaSetDevice(dev);
      const long long l0 = launch_counter();
      cudaStream_t ws = nullptr;
      if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(fmu);
        if (own_fail.index < 0) own_fail = Failure{jobs[w][0], LIBRPA_E_CUDA, "batch: stream creation failed"};
        return;
      }
      for (size_t k = w; k < jobs.size(); k += nwk) {
        const std::vector<int> &job = jobs[k];
        int at = 0;   // position in the job of the handle an error concerns
        try {
          if (job.size() == 1 && !chi0_fits_tc_batch(*hs[job[0]])) {
            run_own(*hs[job[0]], ws, &ec[job[0]]);
          } else {
            std::vector<Handle *> g;
            std::vector<double *> out;
            for (int i : job) {
              g.push_back(hs[i]);
              out.push_back(&ec[i]);
            }
            run_tc_group(g, ws, out.data(), &at);
          }
        } catch (const Error &e) {
          cudaStreamSynchronize(ws);
          std::lock_guard<std::mutex> lk(fmu);
          if (own_fail.index < 0) own_fail = Failure{job[at], e.code, e.msg};
        } catch (const std::bad_alloc &) {
          std::lock_guard<std::mutex> lk(fmu);
          if (own_fail.index < 0) own_fail = Failure{job[at], LIBRPA_E_NOMEM, "batch: host allocation failed"};
        }
      }
      cudaStreamSynchronize(ws);
      cudaStreamDestroy(ws);
      std::lock_guard<std::mutex> lk(fmu);
      own_launches += launch_counter() - l0;
    });
  // merged handles on the first merged handle's stream (this thread)
  Failure main_fail;
  bool replay = false;
  float t[4] = {0, 0, 0, 0};
  long long main_launches = 0;
  std::vector<librpa_gpu *> mh;
  for (int i : mi) mh.push_back(hs[i]);
  if (!mh.empty()) {
    StreamSwap swap(mh);
    cudaStream_t s = mh[0]->stream;
    int cur = 0;
    cudaEvent_t ev[5] = {}, ev_chi0 = nullptr;
    try {
      for (auto &e : ev) LR_CUDA(cudaEventCreate(&e));
      LR_CUDA(cudaEventCreate(&ev_chi0));
      const long long l0 = launch_counter();
      LR_CUDA(cudaEventRecord(ev[0], s));
      std::vector<double> imag(mh.size());
      for (cur = 0; cur < (int)mh.size(); ++cur) {
        materialize(*mh[cur]);
        mh[cur]->stats = librpa_gpu_stats{};
        imag[cur] = green_build(*mh[cur]);
      }
      LR_CUDA(cudaEventRecord(ev[1], s));
      std::vector<Handle *> merged;
      for (cur = 0; cur < (int)mh.size(); ++cur) {
        Handle &h = *mh[cur];
        if (h.lri_dirty) {
          chi0_plan(h);
          h.lri_dirty = false;
        }
        merged.push_back(&h);
      }
      cur = 0;
      replay = chi0_run_merged(merged, b->m);
      LR_CUDA(cudaEventRecord(ev_chi0, s));
      // per handle: transforms and ln det, then its chi0(q, i omega) and workspace are released,
      // so the batch holds every chi0(R, tau) but one handle's transient buffers at a time
      for (cur = 0; cur < (int)mh.size(); ++cur) {
        Handle &h = *mh[cur];
        LR_CUDA(cudaEventRecord(ev[2], s));
        freq_transform(h);
        h.chi0_done = true;
        LR_CUDA(cudaEventRecord(ev[3], s));
        const int rc = ec_run(h, &ec[mi[cur]], nullptr, nullptr);
        if (rc == LIBRPA_E_NOT_PD) throw Error{rc, "ec: a Cholesky pivot was <= 0"};
        if (rc) throw Error{rc, "ec: a bounded device wait ran out"};
        LR_CUDA(cudaEventRecord(ev[4], s));
        LR_CUDA(cudaEventSynchronize(ev[4]));
        float a = 0, c = 0;
        cudaEventElapsedTime(&a, ev[2], ev[3]);
        cudaEventElapsedTime(&c, ev[3], ev[4]);
        t[2] += a;
        t[3] += c;
        h.release(h.d_chi_qw);
        h.release(h.work);
        h.chi0_done = false;   // chi0(q, i omega) is gone: ec needs a new chi0
      }
      LR_CUDA(cudaStreamSynchronize(s));
      cudaEventElapsedTime(&t[0], ev[0], ev[1]);
      cudaEventElapsedTime(&t[1], ev[1], ev_chi0);
      for (librpa_gpu *h : mh) h->resolve_timers();
      for (cur = 0; cur < (int)mh.size(); ++cur)
        if (mh[cur]->opts.check_level >= 1 && !(imag[cur] <= 1e-10))
          throw Error{LIBRPA_E_NUMERIC, "batch: G(R, tau) has an imaginary part"};
      main_launches = launch_counter() - l0;
    } catch (const Error &e) {
      cudaStreamSynchronize(s);
      main_fail = Failure{mi[std::min(cur, (int)mi.size() - 1)], e.code, e.msg};
    } catch (const std::bad_alloc &) {
      main_fail = Failure{mi[std::min(cur, (int)mi.size() - 1)], LIBRPA_E_NOMEM, "batch: host allocation failed"};
    }
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
    if (ev_chi0) cudaEventDestroy(ev_chi0);
  }
  for (std::thread &w : workers) w.join();
  if (main_fail.index >= 0) return fail_at(main_fail.index, main_fail.code, main_fail.msg);
  if (own_fail.index >= 0) return fail_at(own_fail.index, own_fail.code, own_fail.msg);
  b->st.n_merged = (int)mi.size();
  b->st.n_merged_tc = n_tc_merged;
  b->st.graph = replay ? 1 : 0;
  b->st.var_nx = b->m.var_nx;
  b->st.var_fin = b->m.var_fin;
  b->st.ms_green = t[0];
  b->st.ms_chi0 = t[1];
  b->st.ms_freq = t[2];
  b->st.ms_ec = t[3];
  b->st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  b->st.launches = main_launches + own_launches;
  return LIBRPA_OK;
}

int librpa_gpu_batch_get_stats(librpa_gpu_batch_t b, librpa_gpu_batch_stats *st) {
  if (!b || !st) return LIBRPA_E_ARG;
  *st = b->st;
  return LIBRPA_OK;
}

void librpa_gpu_batch_destroy(librpa_gpu_batch_t b) {
  if (!b) return;
  cudaSetDevice(b->hs[0]->opts.device);
  cudaStreamSynchronize(b->hs[0]->stream);
  b->m.reset();
  Handle *owner = b->m.hs.empty() ? b->hs[0] : b->m.hs[0];   // the descriptors were allocated through it
  for (DevBuf &d : b->m.nx_args) owner->release(d);
  for (DevBuf &d : b->m.fin_args) owner->release(d);
  delete b;
}

}  // extern "C"
