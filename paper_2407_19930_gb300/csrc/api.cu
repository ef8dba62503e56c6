// C ABI of librpa_gpu: argument checking, host staging, device memory and the call
// sequence of the response-function and correlation-energy path (Sec. 2 of the paper).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <new>

#include "internal.h"

namespace librpa {

long long &launch_counter() {
  static thread_local long long n = 0;   // per host thread: every handle runs on one thread at a time
  return n;
}

void *Handle::dalloc(size_t bytes) {
  if (bytes == 0) return nullptr;
  if (opts.hbm_budget && bytes_held + bytes > opts.hbm_budget)
    throw Error{LIBRPA_E_NOMEM, "allocation of " + std::to_string(bytes) + " bytes exceeds the HBM budget (" +
                                    std::to_string(opts.hbm_budget) + " bytes, " + std::to_string(bytes_held) +
                                    " held)"};
  void *p = nullptr;
  if (opts.dev_alloc) {
    p = opts.dev_alloc(bytes, opts.alloc_ctx);
    if (!p) throw Error{LIBRPA_E_NOMEM, "device allocator hook returned NULL for " + std::to_string(bytes) + " bytes"};
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{LIBRPA_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    }
  }
  allocs[p] = bytes;
  bytes_held += bytes;
  bytes_peak = std::max(bytes_peak, bytes_held);
  return p;
}

void Handle::dfree(void *p) {
  if (!p) return;
  auto it = allocs.find(p);
  if (it != allocs.end()) {
    bytes_held -= it->second;
    allocs.erase(it);
  }
  if (opts.dev_free)
    opts.dev_free(p, opts.alloc_ctx);
  else
    cudaFree(p);
}

void Handle::ensure(DevBuf &b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return;
  release(b);
  b.p = dalloc(bytes);
  b.bytes = bytes;
}

void Handle::release(DevBuf &b) {
  if (b.p) {
    // work queued on the stream may still read the buffer
    cudaStreamSynchronize(stream);
    dfree(b.p);
  }
  b.p = nullptr;
  b.bytes = 0;
}

void Handle::upload_async(DevBuf &dst, const void *src, size_t bytes) {
  ensure(dst, std::max<size_t>(bytes, 1));
  if (!bytes) return;
  const size_t need = (bytes + 255) / 256 * 256;
  if (need > pin_bytes) {   // grow: wait for every copy from the old ring, then replace it
    if (pin_done) LR_CUDA(cudaEventSynchronize(pin_done));
    if (pin) cudaFreeHost(pin);
    pin = nullptr;
    pin_bytes = std::max(need, (size_t)32 << 20);
    LR_CUDA(cudaMallocHost(&pin, pin_bytes));
    pin_head = 0;
  } else if (pin_head + need > pin_bytes || (pin_stream && pin_stream != stream)) {
    if (pin_done) LR_CUDA(cudaEventSynchronize(pin_done));
    pin_head = 0;
  }
  if (!pin_done) LR_CUDA(cudaEventCreateWithFlags(&pin_done, cudaEventDisableTiming));
  std::memcpy(pin + pin_head, src, bytes);
  LR_CUDA(cudaMemcpyAsync(dst.p, pin + pin_head, bytes, cudaMemcpyHostToDevice, stream));
  LR_CUDA(cudaEventRecord(pin_done, stream));
  pin_stream = stream;
  pin_head += need;
}

void Handle::free_pinned() {
  if (pin_done) {
    cudaEventSynchronize(pin_done);
    cudaEventDestroy(pin_done);
  }
  if (pin) cudaFreeHost(pin);
  pin = nullptr;
  pin_done = nullptr;
  pin_bytes = pin_head = 0;
  pin_stream = nullptr;
}

void Handle::resolve_timers() {
  for (auto &t : timed) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      if (t.kind == 0) {
        stats.ms_gemm_chi0 += ms;
        stats.flop_gemm_chi0 += t.flops;
        stats.flop_exec_gemm_chi0 += t.exec_flops;
        stats.n_gemm_chi0 += 1;
      } else {
        stats.ms_gemm_ec += ms;
        stats.flop_gemm_ec += t.flops;
        stats.flop_exec_gemm_ec += t.exec_flops;
        stats.n_gemm_ec += 1;
      }
    }
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  timed.clear();
}

namespace {

int fail(Handle *h, int code, const std::string &msg) {
  if (h) h->last_error = msg;
  return code;
}

template <class F>
int guarded(Handle *h, F &&f) {
  if (!h) return LIBRPA_E_ARG;
  h->last_error.clear();
  try {
    int rc = f();
    return rc;
  } catch (const Error &e) {
    return fail(h, e.code, e.msg);
  } catch (const std::bad_alloc &) {
    return fail(h, LIBRPA_E_NOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(h, LIBRPA_E_ARG, e.what());
  }
}

void free_device_state(Handle &h) {
  h.release(h.d_g);
  h.release(h.d_chi_tau);
  h.release(h.d_chi_qw);
  h.release(h.d_cpack);
  h.release(h.d_vq);
  h.release(h.d_wfc);
  h.release(h.d_eig);
  h.release(h.d_occ);
  h.release(h.zgemm_args);
  h.release(h.rgemm_args);
  h.release(h.gemm_args);
  h.release(h.oz_args);
  h.release(h.work);
  h.release(h.d_gmask);
  h.release(h.d_screen_tab);
  for (DevBuf *b : h.plan.all()) h.release(*b);
  h.lri_dirty = true;
}

}  // namespace

void release_device(Handle &h) { free_device_state(h); }

void materialize(Handle &h) {
  if (!h.deferred) return;
  const size_t nq = h.mesh.size(), nk = (size_t)h.nspins * nq, nb = h.nao, per_k = nb * h.nao,
               n2 = (size_t)h.naux * h.naux;
  if (!h.d_wfc.p && !h.stage_wfc.empty()) {
    h.ensure(h.d_wfc, nk * per_k * 16);
    h.ensure(h.d_eig, nk * nb * 8);
    h.ensure(h.d_occ, nk * nb * 8);
    LR_CUDA(cudaMemcpyAsync(h.d_wfc.p, h.stage_wfc.data(), nk * per_k * 16, cudaMemcpyHostToDevice, h.stream));
    LR_CUDA(cudaMemcpyAsync(h.d_eig.p, h.eig.data(), nk * nb * 8, cudaMemcpyHostToDevice, h.stream));
    LR_CUDA(cudaMemcpyAsync(h.d_occ.p, h.occ.data(), nk * nb * 8, cudaMemcpyHostToDevice, h.stream));
  }
  if (!h.d_vq.p && !h.stage_vq.empty()) {
    h.ensure(h.d_vq, n2 * 16 * nq);
    LR_CUDA(cudaMemcpyAsync(h.d_vq.p, h.stage_vq.data(), n2 * 16 * nq, cudaMemcpyHostToDevice, h.stream));
  }
  LR_CUDA(cudaStreamSynchronize(h.stream));
}

size_t estimate_device_bytes(Handle &h) {
  const int ntau_saved = h.ntau;
  if (!h.have_grid) h.ntau = h.opts.n_tau;
  const size_t nk = h.mesh.size(), ns = h.nspins, nb = h.nao, n2ao = (size_t)h.nao * h.nao,
               n2 = (size_t)h.naux * h.naux;
  size_t b = ns * (nk * nb * h.nao * 16 + 2 * nk * nb * 8);       // KS data
  b += nk * n2 * 16;                                              // V(q)
  b += ns * 2 * (size_t)h.ntau * nk * n2ao * 8;                   // G^occ, G^vir per spin
  b += nk * (size_t)h.ntau * n2 * 16;                             // chi0(q, i omega)
  Chi0Plan P;
  chi0_shape(h, P);
  b += chi0_device_bytes(h, P);
  b += std::max(green_work_bytes(h), std::max(freq_work_bytes(h), ec_work_bytes(h)));
  b += (size_t)64 << 20;                                          // descriptor and tile uploads
  if (h.g_screen > 0)                                             // block mask, atom tables
    b += ns * 2 * (size_t)h.ntau * nk * h.natoms * h.natoms + 8 * (size_t)h.natoms + 512;
  h.ntau = ntau_saved;
  return b;
}

int chi0_prepare(Handle &h) {
  if (!h.have_structure) return fail(&h, LIBRPA_E_STATE, "chi0 before set_structure");
  for (size_t k = 0; k < h.have_k.size(); ++k)
    if (!h.have_k[k])
      return fail(&h, LIBRPA_E_STATE, "chi0: set_green missing for spin " + std::to_string(k / h.mesh.size()) +
                                          ", k index " + std::to_string(k % h.mesh.size()));
  {
    std::vector<char> seen(h.natoms, 0);
    for (auto &kv : h.lri) seen[std::get<0>(kv.first)] = 1;
    for (int a = 0; a < h.natoms; ++a)
      if (!seen[a]) return fail(&h, LIBRPA_E_STATE, "chi0: no LRI block for atom " + std::to_string(a));
  }
  for (size_t k = 1; k < h.efermi_k.size(); ++k)
    if (h.efermi_k[k] != h.efermi_k[0])
      return fail(&h, LIBRPA_E_ARG, "chi0: efermi differs between k points or spins");
  cudaSetDevice(h.opts.device);
  if (!h.have_grid) {
    // transition-energy range of the KS spectrum, within each spin channel: smallest virtual
    // minus largest occupied energy, and largest virtual minus smallest occupied energy
    const int nb = h.nao, nk = h.mesh.size();
    double dmin = 1e300, dmax = -1e300;
    for (int sp = 0; sp < h.nspins; ++sp) {
      double eo_max = -1e300, eo_min = 1e300, ev_min = 1e300, ev_max = -1e300;
      for (int k = 0; k < nk; ++k)
        for (int n = 0; n < nb; ++n) {
          const size_t x = ((size_t)sp * nk + k) * nb + n;
          const double e = h.eig[x], f = h.occ[x];
          if (f > 0) { eo_max = std::fmax(eo_max, e); eo_min = std::fmin(eo_min, e); }
          if (f < 1) { ev_min = std::fmin(ev_min, e); ev_max = std::fmax(ev_max, e); }
        }
      if (eo_max < -1e299 || ev_min > 1e299) continue;   // no transitions in this channel
      dmin = std::fmin(dmin, ev_min - eo_max);
      dmax = std::fmax(dmax, ev_max - eo_min);
    }
    if (!(dmin > 0) || dmin > 1e299)
      return fail(&h, LIBRPA_E_ARG, "chi0: no gap between occupied and virtual states");
    int n = h.opts.n_tau;
    h.tau.resize(n);
    h.omega.resize(n);
    h.w_omega.resize(n);
    h.gamma.resize((size_t)n * n);
    int rc = h.opts.grid_kind == LIBRPA_GRID_GAUSS_LEGENDRE
                 ? build_grid(n, dmin, dmax, h.tau.data(), h.omega.data(), h.w_omega.data(), h.gamma.data())
                 : build_grid_minimax(n, dmin, dmax, h.tau.data(), h.omega.data(), h.w_omega.data(),
                                      h.gamma.data(), nullptr);
    if (rc) return fail(&h, rc, "chi0: grid construction failed");
    h.ntau = n;
    h.have_grid = true;
  }
  return LIBRPA_OK;
}

}  // namespace librpa

using namespace librpa;


extern "C" {

void librpa_gpu_default_opts(librpa_gpu_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->device = 0;
  o->n_tau = 16;
  o->precision = LIBRPA_FP64;
  o->check_level = 1;
  o->grid_kind = LIBRPA_GRID_MINIMAX;
}

int librpa_gpu_create(librpa_gpu_t *hp, const librpa_gpu_opts *o) {
  if (!hp || !o) return LIBRPA_E_ARG;
  *hp = nullptr;
  if (o->n_tau < 1 || o->n_tau > 64 || o->precision < LIBRPA_FP64 || o->precision > LIBRPA_SPLIT_FAST ||
      o->chi0_slices < 0 || o->chi0_slices > 5 || o->ec_slices < 0 || o->ec_slices > 5 || o->test_stall_gemms < 0 ||
      (o->grid_kind != LIBRPA_GRID_MINIMAX && o->grid_kind != LIBRPA_GRID_GAUSS_LEGENDRE) ||
      (o->grid_kind == LIBRPA_GRID_MINIMAX && o->n_tau > kMinimaxMaxN))
    return LIBRPA_E_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return LIBRPA_E_CUDA;
  }
  if (o->device < 0 || o->device >= ndev) return LIBRPA_E_ARG;
  librpa_gpu *h = new (std::nothrow) librpa_gpu();
  if (!h) return LIBRPA_E_NOMEM;
  h->opts = *o;
  h->stalls_left = o->test_stall_gemms;
  {
    // arithmetic per stage (-1 = FP64 pipes, 0 = plain BF16, 1..5 = digit planes, 6 = plain
    // TF32, 7 = 3xTF32): presets, then explicit overrides
    static const int chi0_preset[7] = {-1, 5, 3, 0, 6, 7, 3}, ec_preset[7] = {-1, 5, 5, 5, 5, 5, 4};
    h->chi0_S = o->chi0_slices ? o->chi0_slices : chi0_preset[o->precision];
    h->ec_S = o->ec_slices ? o->ec_slices : ec_preset[o->precision];
    h->freq_f32 = o->precision == LIBRPA_SPLIT_FAST;
  }
  if (cudaSetDevice(o->device) != cudaSuccess) {
    delete h;
    return LIBRPA_E_CUDA;
  }
  if (o->stream) {
    h->stream = (cudaStream_t)o->stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return LIBRPA_E_CUDA;
    }
    h->own_stream = true;
  }
  *hp = h;
  return LIBRPA_OK;
}

int librpa_gpu_set_structure(librpa_gpu_t h, int natoms, const double lat[9], const double *pos,
                             const int *n_ao, const int *n_aux, int nk1, int nk2, int nk3, int nspins,
                             double r_cut) {
  return guarded(h, [&]() -> int {
    if (natoms < 1 || !lat || !pos || !n_ao || !n_aux || nk1 < 1 || nk2 < 1 || nk3 < 1 || !(r_cut > 0))
      return fail(h, LIBRPA_E_ARG, "set_structure: bad dimensions or NULL arrays");
    if (nspins != 1 && nspins != 2) return fail(h, LIBRPA_E_ARG, "set_structure: nspins must be 1 or 2");
    for (int a = 0; a < natoms; ++a)
      if (n_ao[a] < 1 || n_ao[a] > 64 || n_aux[a] < 1 || n_aux[a] > 256)
        return fail(h, LIBRPA_E_ARG, "set_structure: n_ao must be 1..64 and n_aux 1..256 per atom");
    cudaSetDevice(h->opts.device);
    free_device_state(*h);
    h->natoms = natoms;
    h->nspins = nspins;
    std::memcpy(h->lat, lat, sizeof(double) * 9);
    h->pos.assign(pos, pos + 3 * natoms);
    h->n_ao.assign(n_ao, n_ao + natoms);
    h->n_aux.assign(n_aux, n_aux + natoms);
    h->ao_off.assign(natoms + 1, 0);
    h->aux_off.assign(natoms + 1, 0);
    for (int a = 0; a < natoms; ++a) {
      h->ao_off[a + 1] = h->ao_off[a] + n_ao[a];
      h->aux_off[a + 1] = h->aux_off[a] + n_aux[a];
    }
    h->nao = h->ao_off[natoms];
    h->naux = h->aux_off[natoms];
    h->mesh = Mesh{nk1, nk2, nk3};
    h->r_cut = r_cut;
    const int nk = h->mesh.size();
    h->lri.clear();
    h->wq.clear();
    h->stage_wfc.clear();
    h->stage_vq.clear();
    h->eig.assign((size_t)nspins * nk * h->nao, 0.0);
    h->occ.assign((size_t)nspins * nk * h->nao, 0.0);
    h->have_k.assign((size_t)nspins * nk, 0);
    h->efermi_k.assign((size_t)nspins * nk, 0.0);
    h->have_q.assign(nk, 0);
    h->have_grid = h->grid_user = false;
    h->chi0_done = false;
    h->lri_dirty = true;
    h->have_structure = true;
    return LIBRPA_OK;
  });
}

int librpa_gpu_set_lri_coeffs(librpa_gpu_t h, int I, int K, const int R[3], const double *C) {
  return guarded(h, [&]() -> int {
    if (!h->have_structure) return fail(h, LIBRPA_E_STATE, "set_lri_coeffs before set_structure");
    if (I < 0 || I >= h->natoms || K < 0 || K >= h->natoms || !R || !C)
      return fail(h, LIBRPA_E_ARG, "set_lri_coeffs: bad atom index or NULL");
    double d2 = 0;
    for (int x = 0; x < 3; ++x) {
      double v = h->pos[3 * K + x] - h->pos[3 * I + x];
      for (int a = 0; a < 3; ++a) v += R[a] * h->lat[3 * a + x];
      d2 += v * v;
    }
    if (std::sqrt(d2) > h->r_cut * (1 + 1e-12))
      return fail(h, LIBRPA_E_ARG, "set_lri_coeffs: atoms farther apart than r_cut");
    size_t n = (size_t)h->n_aux[I] * h->n_ao[I] * h->n_ao[K];
    h->lri[std::make_tuple(I, K, R[0], R[1], R[2])] = std::vector<double>(C, C + n);
    h->lri_dirty = true;
    h->chi0_done = false;
    return LIBRPA_OK;
  });
}

int librpa_gpu_set_green(librpa_gpu_t h, int ispin, int ik, int nbands, const double *eig, const double *occ,
                         const double *wfc_re, const double *wfc_im, double efermi) {
  return guarded(h, [&]() -> int {
    if (!h->have_structure) return fail(h, LIBRPA_E_STATE, "set_green before set_structure");
    if (ispin < 0 || ispin >= h->nspins || ik < 0 || ik >= h->mesh.size() || nbands != h->nao || !eig || !occ ||
        !wfc_re || !wfc_im)
      return fail(h, LIBRPA_E_ARG, "set_green: bad spin/k index, nbands != n_ao total, or NULL");
    const int nb = h->nao;
    const size_t sk = (size_t)ispin * h->mesh.size() + ik;   // (spin, k) slot
    for (int n = 0; n < nb; ++n) {
      if (!(occ[n] >= 0.0 && occ[n] <= 1.0) || !std::isfinite(eig[n]))
        return fail(h, LIBRPA_E_ARG, "set_green: occupations must be in [0, 1] and energies finite");
      h->eig[sk * nb + n] = eig[n];
      h->occ[sk * nb + n] = occ[n];
    }
    const size_t nk = (size_t)h->nspins * h->mesh.size(), per_k = (size_t)nb * h->nao;
    if (h->deferred) {   // kept on the host until the request is admitted
      h->stage_wfc.resize(nk * per_k * 2);
      double *w = h->stage_wfc.data() + sk * per_k * 2;
      for (size_t x = 0; x < per_k; ++x) {
        w[2 * x] = wfc_re[x];
        w[2 * x + 1] = wfc_im[x];
      }
      h->efermi_k[sk] = efermi;
      h->have_k[sk] = 1;
      h->chi0_done = false;
      return LIBRPA_OK;
    }
    cudaSetDevice(h->opts.device);
    h->ensure(h->d_wfc, nk * per_k * 16);
    h->ensure(h->d_eig, nk * nb * 8);
    h->ensure(h->d_occ, nk * nb * 8);
    std::vector<double> w(2 * per_k);
    for (size_t x = 0; x < per_k; ++x) {
      w[2 * x] = wfc_re[x];
      w[2 * x + 1] = wfc_im[x];
    }
    LR_CUDA(cudaMemcpyAsync((char *)h->d_wfc.p + sk * per_k * 16, w.data(), per_k * 16, cudaMemcpyHostToDevice,
                            h->stream));
    LR_CUDA(cudaMemcpyAsync((double *)h->d_eig.p + sk * nb, h->eig.data() + sk * nb, nb * 8,
                            cudaMemcpyHostToDevice, h->stream));
    LR_CUDA(cudaMemcpyAsync((double *)h->d_occ.p + sk * nb, h->occ.data() + sk * nb, nb * 8,
                            cudaMemcpyHostToDevice, h->stream));
    LR_CUDA(cudaStreamSynchronize(h->stream));
    h->efermi_k[sk] = efermi;
    h->have_k[sk] = 1;
    h->chi0_done = false;
    return LIBRPA_OK;
  });
}

int librpa_gpu_set_coulomb(librpa_gpu_t h, int iq, const double *V_re, const double *V_im) {
  return guarded(h, [&]() -> int {
    if (!h->have_structure) return fail(h, LIBRPA_E_STATE, "set_coulomb before set_structure");
    if (iq < 0 || iq >= h->mesh.size() || !V_re || !V_im) return fail(h, LIBRPA_E_ARG, "set_coulomb: bad q or NULL");
    const size_t n2 = (size_t)h->naux * h->naux;
    if (h->deferred) {   // kept on the host until the request is admitted
      h->stage_vq.resize(n2 * 2 * h->mesh.size());
      double *v = h->stage_vq.data() + (size_t)iq * n2 * 2;
      for (size_t x = 0; x < n2; ++x) {
        v[2 * x] = V_re[x];
        v[2 * x + 1] = V_im[x];
      }
      h->have_q[iq] = 1;
      h->vq_sym = h->vq_real = -1;
      return LIBRPA_OK;
    }
    cudaSetDevice(h->opts.device);
    h->ensure(h->d_vq, n2 * 16 * h->mesh.size());
    std::vector<double> tmp(2 * n2);
    for (size_t x = 0; x < n2; ++x) {
      tmp[2 * x] = V_re[x];
      tmp[2 * x + 1] = V_im[x];
    }
    LR_CUDA(cudaMemcpyAsync((char *)h->d_vq.p + n2 * 16 * iq, tmp.data(), n2 * 16, cudaMemcpyHostToDevice,
                            h->stream));
    LR_CUDA(cudaStreamSynchronize(h->stream));
    h->have_q[iq] = 1;
    h->vq_sym = h->vq_real = -1;
    return LIBRPA_OK;
  });
}

int librpa_gpu_set_grid(librpa_gpu_t h, int ntau, const double *tau, int nomega, const double *omega,
                        const double *w_omega, const double *gamma) {
  return guarded(h, [&]() -> int {
    if (!h->have_structure) return fail(h, LIBRPA_E_STATE, "set_grid before set_structure");
    if (ntau < 1 || ntau > 64 || nomega != ntau || !tau || !omega || !w_omega || !gamma)
      return fail(h, LIBRPA_E_ARG, "set_grid: need ntau == nomega in 1..64 and non-NULL arrays");
    h->ntau = ntau;
    h->tau.assign(tau, tau + ntau);
    h->omega.assign(omega, omega + nomega);
    h->w_omega.assign(w_omega, w_omega + nomega);
    h->gamma.assign(gamma, gamma + (size_t)nomega * ntau);
    h->have_grid = h->grid_user = true;
    h->chi0_done = false;
    return LIBRPA_OK;
  });
}

int librpa_gpu_set_q_weights(librpa_gpu_t h, const double *w) {
  return guarded(h, [&]() -> int {
    if (!h->have_structure) return fail(h, LIBRPA_E_STATE, "set_q_weights before set_structure");
    if (!w) {
      h->wq.clear();
      return LIBRPA_OK;
    }
    const int nq = h->mesh.size();
    bool any = false;
    for (int q = 0; q < nq; ++q) {
      if (!(w[q] >= 0.0) || !std::isfinite(w[q]))
        return fail(h, LIBRPA_E_ARG, "set_q_weights: weights must be finite and >= 0");
      any = any || w[q] > 0.0;
    }
    if (!any) return fail(h, LIBRPA_E_ARG, "set_q_weights: at least one weight must be > 0");
    h->wq.assign(w, w + nq);
    return LIBRPA_OK;
  });
}

int librpa_gpu_set_screening(librpa_gpu_t h, double threshold) {
  return guarded(h, [&]() -> int {
    if (!(threshold >= 0.0) || !std::isfinite(threshold))
      return fail(h, LIBRPA_E_ARG, "set_screening: threshold must be finite and >= 0");
    h->g_screen = threshold;
    h->chi0_done = false;
    return LIBRPA_OK;
  });
}

int librpa_gpu_build_grid(int n, double dmin, double dmax, double *tau, double *omega, double *w_omega,
                          double *gamma) {
  try {
    return librpa::build_grid(n, dmin, dmax, tau, omega, w_omega, gamma);
  } catch (...) {
    return LIBRPA_E_NOMEM;
  }
}

int librpa_gpu_build_grid_minimax(int n, double dmin, double dmax, double *tau, double *omega, double *w_omega,
                                  double *gamma, double *info) {
  try {
    return librpa::build_grid_minimax(n, dmin, dmax, tau, omega, w_omega, gamma, info);
  } catch (...) {
    return LIBRPA_E_NOMEM;
  }
}

int librpa_gpu_get_grid(librpa_gpu_t h, int *n, double *tau, double *omega, double *w_omega, double *gamma) {
  return guarded(h, [&]() -> int {
    if (!h->have_grid) return fail(h, LIBRPA_E_STATE, "get_grid: no grid yet");
    if (!n) return fail(h, LIBRPA_E_ARG, "get_grid: NULL n");
    *n = h->ntau;
    if (tau) std::memcpy(tau, h->tau.data(), sizeof(double) * h->ntau);
    if (omega) std::memcpy(omega, h->omega.data(), sizeof(double) * h->ntau);
    if (w_omega) std::memcpy(w_omega, h->w_omega.data(), sizeof(double) * h->ntau);
    if (gamma) std::memcpy(gamma, h->gamma.data(), sizeof(double) * h->ntau * h->ntau);
    return LIBRPA_OK;
  });
}

int librpa_gpu_chi0(librpa_gpu_t h, double *out_re, double *out_im) {
  return guarded(h, [&]() -> int {
    if (int rc = chi0_prepare(*h)) return rc;
    materialize(*h);
    h->stats = librpa_gpu_stats{};
    long long l0 = launch_counter();
    cudaEvent_t ev[4];
    for (auto &e : ev) LR_CUDA(cudaEventCreate(&e));
    LR_CUDA(cudaEventRecord(ev[0], h->stream));
    double imag = green_build(*h);
    LR_CUDA(cudaEventRecord(ev[1], h->stream));
    if (h->lri_dirty) {
      chi0_plan(*h);
      h->lri_dirty = false;
    }
    double ms_gemm = 0;
    chi0_run(*h, &ms_gemm);
    LR_CUDA(cudaEventRecord(ev[2], h->stream));
    freq_transform(*h);
    LR_CUDA(cudaEventRecord(ev[3], h->stream));
    LR_CUDA(cudaStreamSynchronize(h->stream));
    float t;
    cudaEventElapsedTime(&t, ev[0], ev[1]);
    h->stats.ms_green = t;
    cudaEventElapsedTime(&t, ev[1], ev[2]);
    h->stats.ms_chi0 = t;
    cudaEventElapsedTime(&t, ev[2], ev[3]);
    h->stats.ms_freq = t;
    for (auto &e : ev) cudaEventDestroy(e);
    h->resolve_timers();
    h->stats.flop_chi0 = h->flop_chi0_run;
    h->stats.launches = launch_counter() - l0;
    h->stats.bytes_device = h->bytes_held;
    h->stats.bytes_device_peak = h->bytes_peak;
    if (h->opts.check_level >= 1 && !(imag <= 1e-10))
      return fail(h, LIBRPA_E_NUMERIC, "chi0: G(R, tau) has a relative imaginary part of " + std::to_string(imag) +
                                           " (inputs without time-reversal symmetry?)");
    h->chi0_done = true;
    if (out_re || out_im) {
      const size_t n2 = (size_t)h->naux * h->naux, tot = n2 * h->mesh.size() * h->ntau;
      std::vector<double> tmp(2 * n2);
      for (size_t s = 0; s < tot / n2; ++s) {
        LR_CUDA(cudaMemcpy(tmp.data(), (const char *)h->d_chi_qw.p + s * n2 * 16, n2 * 16, cudaMemcpyDeviceToHost));
        for (size_t x = 0; x < n2; ++x) {
          if (out_re) out_re[s * n2 + x] = tmp[2 * x];
          if (out_im) out_im[s * n2 + x] = tmp[2 * x + 1];
        }
      }
    }
    return LIBRPA_OK;
  });
}

int librpa_gpu_ec(librpa_gpu_t h, double *ec, double *ec_q, double *ec_w) {
  return guarded(h, [&]() -> int {
    if (!h->chi0_done) return fail(h, LIBRPA_E_STATE, "ec before a successful chi0");
    if (!ec) return fail(h, LIBRPA_E_ARG, "ec: NULL output");
    for (int q = 0; q < h->mesh.size(); ++q)
      if (!h->have_q[q]) return fail(h, LIBRPA_E_STATE, "ec: set_coulomb missing for q index " + std::to_string(q));
    cudaSetDevice(h->opts.device);
    long long l0 = launch_counter();
    cudaEvent_t e0, e1;
    LR_CUDA(cudaEventCreate(&e0));
    LR_CUDA(cudaEventCreate(&e1));
    LR_CUDA(cudaEventRecord(e0, h->stream));
    int rc = ec_run(*h, ec, ec_q, ec_w);
    LR_CUDA(cudaEventRecord(e1, h->stream));
    LR_CUDA(cudaStreamSynchronize(h->stream));
    float t;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->stats.ms_ec = t;
    h->stats.ms_gemm_ec = h->stats.flop_gemm_ec = 0;
    h->stats.n_gemm_ec = 0;
    h->resolve_timers();
    h->stats.launches += launch_counter() - l0;
    h->stats.bytes_device = h->bytes_held;
    h->stats.bytes_device_peak = h->bytes_peak;
    if (rc == LIBRPA_E_NOT_PD)
      return fail(h, rc, "ec: a Cholesky pivot was <= 0 (V(q) or 1 - V^1/2 chi0 V^1/2 not positive definite)");
    if (rc == LIBRPA_E_TIMEOUT) return fail(h, rc, "ec: a bounded wait in the tensor-core GEMM ran out");
    return rc;
  });
}

int librpa_gpu_get_green(librpa_gpu_t h, int itau, int iR, double *go, double *gv) {
  return guarded(h, [&]() -> int {
    if (!h->d_g.p) return fail(h, LIBRPA_E_STATE, "get_green: G not computed");
    if (itau < 0 || itau >= h->ntau || iR < 0 || iR >= h->mesh.size())
      return fail(h, LIBRPA_E_ARG, "get_green: index out of range");
    const size_t n2 = (size_t)h->nao * h->nao, slab = n2 * h->ntau * h->mesh.size();
    const size_t off = ((size_t)itau * h->mesh.size() + iR) * n2;
    if (go) LR_CUDA(cudaMemcpy(go, (double *)h->d_g.p + off, n2 * 8, cudaMemcpyDeviceToHost));
    if (gv) LR_CUDA(cudaMemcpy(gv, (double *)h->d_g.p + slab + off, n2 * 8, cudaMemcpyDeviceToHost));
    return LIBRPA_OK;
  });
}

int librpa_gpu_get_chi0_tau(librpa_gpu_t h, int itau, int iR, double *out) {
  return guarded(h, [&]() -> int {
    if (!h->chi0_done) return fail(h, LIBRPA_E_STATE, "get_chi0_tau: chi0 not computed");
    if (itau < 0 || itau >= h->ntau || iR < 0 || iR >= h->mesh.size() || !out)
      return fail(h, LIBRPA_E_ARG, "get_chi0_tau: index out of range or NULL");
    const size_t n2 = (size_t)h->naux * h->naux;
    LR_CUDA(cudaMemcpy(out, (double *)h->d_chi_tau.p + ((size_t)itau * h->mesh.size() + iR) * n2, n2 * 8,
                       cudaMemcpyDeviceToHost));
    return LIBRPA_OK;
  });
}

int librpa_gpu_get_chi0_freq(librpa_gpu_t h, int iq, int iw, double *re, double *im) {
  return guarded(h, [&]() -> int {
    if (!h->chi0_done) return fail(h, LIBRPA_E_STATE, "get_chi0_freq: chi0 not computed");
    if (iq < 0 || iq >= h->mesh.size() || iw < 0 || iw >= h->ntau)
      return fail(h, LIBRPA_E_ARG, "get_chi0_freq: index out of range");
    const size_t n2 = (size_t)h->naux * h->naux;
    std::vector<double> tmp(2 * n2);
    LR_CUDA(cudaMemcpy(tmp.data(), (const char *)h->d_chi_qw.p + ((size_t)iq * h->ntau + iw) * n2 * 16, n2 * 16,
                       cudaMemcpyDeviceToHost));
    for (size_t x = 0; x < n2; ++x) {
      if (re) re[x] = tmp[2 * x];
      if (im) im[x] = tmp[2 * x + 1];
    }
    return LIBRPA_OK;
  });
}

int librpa_gpu_set_green_dev(librpa_gpu_t h, int ispin, int ik, int nbands, const double *eig, const double *occ,
                             const double *wfc, double efermi) {
  return guarded(h, [&]() -> int {
    if (!h->have_structure) return fail(h, LIBRPA_E_STATE, "set_green_dev before set_structure");
    if (h->deferred) return fail(h, LIBRPA_E_STATE, "set_green_dev on a request handle (inputs stay on the host)");
    if (ispin < 0 || ispin >= h->nspins || ik < 0 || ik >= h->mesh.size() || nbands != h->nao || !eig || !occ ||
        !wfc || (uintptr_t)wfc % 16)
      return fail(h, LIBRPA_E_ARG, "set_green_dev: bad spin/k index, nbands != n_ao total, NULL or misaligned");
    const int nb = h->nao;
    const size_t sk = (size_t)ispin * h->mesh.size() + ik;
    for (int n = 0; n < nb; ++n) {
      if (!(occ[n] >= 0.0 && occ[n] <= 1.0) || !std::isfinite(eig[n]))
        return fail(h, LIBRPA_E_ARG, "set_green_dev: occupations must be in [0, 1] and energies finite");
      h->eig[sk * nb + n] = eig[n];
      h->occ[sk * nb + n] = occ[n];
    }
    cudaSetDevice(h->opts.device);
    const size_t nk = (size_t)h->nspins * h->mesh.size(), per_k = (size_t)nb * h->nao;
    h->ensure(h->d_wfc, nk * per_k * 16);
    h->ensure(h->d_eig, nk * nb * 8);
    h->ensure(h->d_occ, nk * nb * 8);
    LR_CUDA(cudaMemcpyAsync((char *)h->d_wfc.p + sk * per_k * 16, wfc, per_k * 16, cudaMemcpyDeviceToDevice,
                            h->stream));
    LR_CUDA(cudaMemcpyAsync((double *)h->d_eig.p + sk * nb, h->eig.data() + sk * nb, nb * 8,
                            cudaMemcpyHostToDevice, h->stream));
    LR_CUDA(cudaMemcpyAsync((double *)h->d_occ.p + sk * nb, h->occ.data() + sk * nb, nb * 8,
                            cudaMemcpyHostToDevice, h->stream));
    h->efermi_k[sk] = efermi;
    h->have_k[sk] = 1;
    h->chi0_done = false;
    return LIBRPA_OK;
  });
}

int librpa_gpu_set_coulomb_dev(librpa_gpu_t h, int iq, const double *V) {
  return guarded(h, [&]() -> int {
    if (!h->have_structure) return fail(h, LIBRPA_E_STATE, "set_coulomb_dev before set_structure");
    if (h->deferred) return fail(h, LIBRPA_E_STATE, "set_coulomb_dev on a request handle (inputs stay on the host)");
    if (iq < 0 || iq >= h->mesh.size() || !V || (uintptr_t)V % 16)
      return fail(h, LIBRPA_E_ARG, "set_coulomb_dev: bad q, NULL or misaligned");
    cudaSetDevice(h->opts.device);
    const size_t n2 = (size_t)h->naux * h->naux;
    h->ensure(h->d_vq, n2 * 16 * h->mesh.size());
    LR_CUDA(cudaMemcpyAsync((char *)h->d_vq.p + n2 * 16 * iq, V, n2 * 16, cudaMemcpyDeviceToDevice, h->stream));
    h->have_q[iq] = 1;
    h->vq_sym = h->vq_real = -1;
    return LIBRPA_OK;
  });
}

int librpa_gpu_get_chi0_freq_dev(librpa_gpu_t h, int iq, int iw, double *out) {
  return guarded(h, [&]() -> int {
    if (!h->chi0_done) return fail(h, LIBRPA_E_STATE, "get_chi0_freq_dev: chi0 not computed");
    if (iq < 0 || iq >= h->mesh.size() || iw < 0 || iw >= h->ntau || !out || (uintptr_t)out % 16)
      return fail(h, LIBRPA_E_ARG, "get_chi0_freq_dev: index out of range, NULL or misaligned output");
    const size_t n2 = (size_t)h->naux * h->naux;
    LR_CUDA(cudaMemcpyAsync(out, (const char *)h->d_chi_qw.p + ((size_t)iq * h->ntau + iw) * n2 * 16, n2 * 16,
                            cudaMemcpyDeviceToDevice, h->stream));
    return LIBRPA_OK;
  });
}

int librpa_gpu_get_stats(librpa_gpu_t h, librpa_gpu_stats *s) {
  if (!h || !s) return LIBRPA_E_ARG;
  *s = h->stats;
  return LIBRPA_OK;
}

const char *librpa_gpu_last_error(librpa_gpu_t h) { return h ? h->last_error.c_str() : "NULL handle"; }

void librpa_gpu_destroy(librpa_gpu_t h) {
  if (!h) return;
  cudaSetDevice(h->opts.device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto &kv : h->allocs) {
    if (h->opts.dev_free)
      h->opts.dev_free(kv.first, h->opts.alloc_ctx);
    else
      cudaFree(kv.first);
  }
  h->allocs.clear();
  h->free_pinned();
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
