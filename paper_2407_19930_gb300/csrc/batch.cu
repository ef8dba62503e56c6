// Batched energies: many independent structures (handles) in one pass on one stream.  The FP64
// chi0 contraction of all handles runs in rounds of point batches, each round's GEMMs as single
// grouped launches over all handles' tiles (uneven block shapes), with tile variants tuned on the
// first run and the launch sequence replayed from a CUDA graph afterwards; handles in the
// tensor-core modes run their own chi0 path in the same pass.  G, the transforms and the
// ln det stage run per handle.
#include <string>
#include <vector>

#include "internal.h"

using namespace librpa;

struct librpa_gpu_batch {
  std::vector<librpa_gpu *> hs;
  MergedChi0 m;
  librpa_gpu_batch_stats st{};
};

namespace {

struct StreamSwap {   // every handle of the batch on hs[0]'s stream for the duration of a run
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
  int cur = 0;
  auto fail_at = [&](int i, int code, const std::string &msg) {
    hs[i]->last_error = msg;
    b->st.failed_index = i;
    return code;
  };
  cudaSetDevice(hs[0]->opts.device);
  for (int i = 0; i < n; ++i) {
    hs[i]->last_error.clear();
    if (int rc = chi0_prepare(*hs[i])) return fail_at(i, rc, hs[i]->last_error);
  }
  StreamSwap swap(hs);
  cudaStream_t s = hs[0]->stream;
  try {
    cudaEvent_t ev[5];
    for (auto &e : ev) LR_CUDA(cudaEventCreate(&e));
    const long long l0 = launch_counter();
    LR_CUDA(cudaEventRecord(ev[0], s));
    std::vector<double> imag(n);
    for (cur = 0; cur < n; ++cur) {
      materialize(*hs[cur]);
      hs[cur]->stats = librpa_gpu_stats{};
      imag[cur] = green_build(*hs[cur]);
    }
    LR_CUDA(cudaEventRecord(ev[1], s));
    std::vector<Handle *> merged;
    for (cur = 0; cur < n; ++cur) {
      Handle &h = *hs[cur];
      if (h.lri_dirty) {
        chi0_plan(h);
        h.lri_dirty = false;
      }
      if (chi0_fits_one_batch(h))
        merged.push_back(&h);
      else
        chi0_run(h, nullptr);
    }
    cur = 0;
    const bool replay = chi0_run_merged(merged, b->m);
    cudaEvent_t ev_chi0;
    LR_CUDA(cudaEventCreate(&ev_chi0));
    LR_CUDA(cudaEventRecord(ev_chi0, s));
    // per handle: transforms and ln det, then its chi0(q, i omega) and workspace are released, so
    // the batch holds every chi0(R, tau) but only one handle's transient buffers at a time
    float t[4] = {0, 0, 0, 0};
    for (cur = 0; cur < n; ++cur) {
      Handle &h = *hs[cur];
      LR_CUDA(cudaEventRecord(ev[2], s));
      freq_transform(h);
      h.chi0_done = true;
      LR_CUDA(cudaEventRecord(ev[3], s));
      const int rc = ec_run(h, &ec[cur], nullptr, nullptr);
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
    cudaEventDestroy(ev_chi0);
    for (auto &e : ev) cudaEventDestroy(e);
    for (librpa_gpu *h : hs) h->resolve_timers();
    for (cur = 0; cur < n; ++cur)
      if (hs[cur]->opts.check_level >= 1 && !(imag[cur] <= 1e-10))
        return fail_at(cur, LIBRPA_E_NUMERIC, "batch: G(R, tau) has an imaginary part");
    b->st.n_merged = (int)merged.size();
    b->st.graph = replay ? 1 : 0;
    b->st.var_nx = b->m.var_nx;
    b->st.var_fin = b->m.var_fin;
    b->st.ms_green = t[0];
    b->st.ms_chi0 = t[1];
    b->st.ms_freq = t[2];
    b->st.ms_ec = t[3];
    b->st.ms_total = t[0] + t[1] + t[2] + t[3];
    b->st.launches = launch_counter() - l0;
  } catch (const Error &e) {
    cudaStreamSynchronize(s);
    return fail_at(cur, e.code, e.msg);
  } catch (const std::bad_alloc &) {
    return fail_at(cur, LIBRPA_E_NOMEM, "batch: host allocation failed");
  }
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
  for (DevBuf &d : b->m.nx_args) b->hs[0]->release(d);
  for (DevBuf &d : b->m.fin_args) b->hs[0]->release(d);
  delete b;
}

}  // extern "C"
