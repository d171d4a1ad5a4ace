// Iterated Conditional Modes driver (Sec. II-D of Scipioni et al., "Kinetic
// Compressive Sensing"): (a) one OS-MAP-OSL-KP pass over all subsets with the
// prior built from the model TACs of the current kinetic maps, then (b) the
// MAP-LM fit of the maps to the new image series.  Everything is issued on one
// stream with no host synchronisation.  Optionally the steady-state iteration
// (prior on) is recorded once into a CUDA graph and replayed, which removes the
// per-launch host cost that dominates small studies.

#include <algorithm>

#include <nvtx3/nvToolsExt.h>

#include "kcs_internal.cuh"

struct kcs_study {
  kcs_study_desc_t d;
  int iterations;
  int use_graph;
  int device;
  cudaStream_t cap;       // private stream the steady-state iteration is captured on
  cudaGraphExec_t exec;   // one ICM iteration with the prior on (null until first use)
  // host I/O of kcs_icm_iterate_host: a private copy stream and its events
  cudaStream_t copy;
  cudaEvent_t ev[4];      // OSL pass done, counts in, fit done, maps out
  std::vector<cudaEvent_t> ev_sub;   // counts rows of subset k in (first upload of a call)
};

using namespace kcs;

namespace {

// (a) one OSL pass over the subsets, (b) the MAP-LM fit, which also refreshes
// F for the next prior; all on stream s, no host synchronisation.
// Huber weight of the fit: the spatial prior is part of KCS only.
float fit_beta_h(const kcs_study_desc_t& d) { return d.method == KCS_METHOD_KCS ? d.beta_h : 0.f; }
int fit_nbhd(const kcs_study_desc_t& d) { return d.neighbourhood == 26 ? 26 : 8; }
// Acceptance threshold of the MAP-LM step: the library default unless given.
float fit_tau(const kcs_study_desc_t& d) { return d.lm_tau_given ? d.lm_tau : KCS_LM_TAU_DEFAULT; }

// wait_sub (optional): one event per subset, waited for before its update.
int issue_osl_pass(const kcs_study* st, bool prior, void* stream,
                   const cudaEvent_t* wait_sub = nullptr) {
  const kcs_study_desc_t& d = st->d;
  const kcs_geometry* g = d.geom;
  if (d.method == KCS_METHOD_INDIRECT) prior = false;
  // host-side ranges (visible in Nsight timelines) around the issue of each phase
  nvtxRangePushA("kcs::osl_pass");
  for (int k = 0; k < g->S; ++k) {
    if (wait_sub && cudaStreamWaitEvent(as_stream(stream), wait_sub[k], 0) != cudaSuccess) {
      nvtxRangePop();
      set_error("cudaStreamWaitEvent failed");
      return KCS_ERR_CUDA;
    }
    const int rc = kcs_osl_update_ex(g, k, d.n_frames, d.frame_dt, d.kappa, d.counts,
                                     d.counts_type, d.randoms, d.randoms_layout, d.bin_factor,
                                     prior ? d.F : nullptr, prior ? d.beta_kp : 0.f,
                                     d.sigma2 > 0.f ? d.sigma2 : 1.f, d.x, d.x_type, d.x_scale,
                                     d.workspace, d.ws_bytes, stream);
    if (rc) {
      nvtxRangePop();
      return rc;
    }
  }
  nvtxRangePop();
  return KCS_OK;
}

// (b) the MAP-LM fit of the maps (and F <- F(params)); nothing for INDIRECT.
int issue_fit(const kcs_study* st, void* stream) {
  const kcs_study_desc_t& d = st->d;
  const kcs_geometry* g = d.geom;
  if (d.method == KCS_METHOD_INDIRECT) return KCS_OK;
  nvtxRangePushA("kcs::map_lm_fit");
  const int rc = kcs_map_lm_fit_nb(d.kin, g->nx, g->ny, g->nz, d.x, d.x_type, d.x_scale, d.params,
                           nullptr, d.n_lm, fit_beta_h(d), d.delta, fit_nbhd(d), fit_tau(d), d.F,
                           d.workspace, d.ws_bytes, stream);
  nvtxRangePop();
  return rc;
}

int issue_iteration(const kcs_study* st, bool prior, void* stream) {
  const int rc = issue_osl_pass(st, prior, stream);
  return rc ? rc : issue_fit(st, stream);
}

// The prior is on once an earlier iteration produced F (or the maps were given).
bool prior_on(const kcs_study* st) {
  return (st->iterations > 0 || st->d.params_given) && st->d.method != KCS_METHOD_INDIRECT;
}

// Record the steady-state iteration once into a CUDA graph.  Capture runs on a
// private non-blocking stream (the caller's may be the legacy default stream,
// which cannot be captured); nothing executes while capturing.
int build_graph(kcs_study* st) {
  if (!st->cap) KCS_CUDA(cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking));
  KCS_CUDA(cudaStreamBeginCapture(st->cap, cudaStreamCaptureModeThreadLocal));
  const int rc = issue_iteration(st, true, st->cap);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st->cap, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  KCS_CUDA(e);
  const cudaError_t ei = cudaGraphInstantiate(&st->exec, graph, 0);
  cudaGraphDestroy(graph);
  KCS_CUDA(ei);
  return KCS_OK;
}

void release_graph(kcs_study* st) {
  if (st->exec) cudaGraphExecDestroy(st->exec);
  st->exec = nullptr;
}

}  // namespace

extern "C" {

size_t kcs_study_workspace_size(const kcs_geometry_t* g, int n_frames) {
  if (!g) return 0;
  return std::max(kcs_osl_workspace_size(g, n_frames), kcs_lm_workspace_size(g->nx, g->ny, g->nz));
}

int kcs_create_study(kcs_study_t** out, const kcs_study_desc_t* d) {
  clear_error();
  KCS_REQUIRE(out && d, "NULL argument");
  KCS_REQUIRE(d->geom && d->kin, "study needs a geometry and a kinetics table");
  KCS_REQUIRE(d->kin->M == d->n_frames, "kinetics has %d frames, study %d", d->kin->M, d->n_frames);
  KCS_REQUIRE(d->frame_dt && d->counts && d->x && d->params && d->F, "NULL device buffer");
  KCS_REQUIRE(d->n_lm >= 0, "n_lm < 0");
  KCS_REQUIRE(d->x_type == KCS_F32 || d->x_type == KCS_BF16 || d->x_type == KCS_F16,
              "x_type %d must be KCS_F32, KCS_BF16 or KCS_F16", d->x_type);
  KCS_REQUIRE(d->counts_type == KCS_F32 || d->counts_type == KCS_U16,
              "counts_type %d must be KCS_F32 or KCS_U16", d->counts_type);
  KCS_REQUIRE(d->method == KCS_METHOD_KCS || d->method == KCS_METHOD_DIRECT ||
                  d->method == KCS_METHOD_INDIRECT,
              "method %d must be KCS_METHOD_KCS, _DIRECT or _INDIRECT", d->method);
  KCS_REQUIRE(!d->lm_tau_given || (d->lm_tau >= 0.f && d->lm_tau < 1.f),
              "lm_tau = %g must lie in [0, 1)", (double)d->lm_tau);
  KCS_REQUIRE(d->neighbourhood == 0 || d->neighbourhood == 8 || d->neighbourhood == 26,
              "neighbourhood %d must be 0, 8 or 26", d->neighbourhood);
  KCS_REQUIRE(d->workspace && d->ws_bytes >= kcs_study_workspace_size(d->geom, d->n_frames),
              "workspace too small (%zu < %zu)", d->ws_bytes,
              kcs_study_workspace_size(d->geom, d->n_frames));
  kcs_study* st = new kcs_study();
  st->d = *d;
  st->iterations = 0;
  st->use_graph = 0;
  st->device = d->geom->device;
  st->cap = nullptr;
  st->exec = nullptr;
  st->copy = nullptr;
  for (auto& e : st->ev) e = nullptr;
  *out = st;
  return KCS_OK;
}

int kcs_destroy_study(kcs_study_t* st) {
  clear_error();
  if (st) {
    release_graph(st);
    if (st->cap) cudaStreamDestroy(st->cap);
    if (st->copy) cudaStreamDestroy(st->copy);
    for (auto e : st->ev)
      if (e) cudaEventDestroy(e);
    for (auto e : st->ev_sub)
      if (e) cudaEventDestroy(e);
  }
  delete st;
  return KCS_OK;
}

int kcs_study_set_graph(kcs_study_t* st, int enable) {
  clear_error();
  KCS_REQUIRE(st, "study is NULL");
  st->use_graph = enable ? 1 : 0;
  if (!enable) release_graph(st);
  return KCS_OK;
}

int kcs_study_iterations(const kcs_study_t* st) { return st ? st->iterations : -1; }

int kcs_study_set_iterations(kcs_study_t* st, int iterations) {
  clear_error();
  KCS_REQUIRE(st, "study is NULL");
  KCS_REQUIRE(iterations >= 0, "iterations < 0");
  st->iterations = iterations;
  return KCS_OK;
}

int kcs_study_fit(kcs_study_t* st, int n_steps, void* stream) {
  clear_error();
  KCS_REQUIRE(st, "study is NULL");
  KCS_REQUIRE(n_steps >= 0, "n_steps < 0");
  const kcs_study_desc_t& d = st->d;
  const kcs_geometry* g = d.geom;
  return kcs_map_lm_fit_nb(d.kin, g->nx, g->ny, g->nz, d.x, d.x_type, d.x_scale, d.params,
                           nullptr, n_steps, fit_beta_h(d), d.delta, fit_nbhd(d), fit_tau(d), d.F,
                           d.workspace, d.ws_bytes, stream);
}

int kcs_icm_iterate(kcs_study_t* st, int n_iter, void* stream) {
  clear_error();
  KCS_REQUIRE(st, "study is NULL");
  KCS_REQUIRE(n_iter >= 0, "n_iter < 0");
  const kcs_study_desc_t& d = st->d;
  const long long V = (long long)d.geom->nz * d.geom->ny * d.geom->nx;
  cudaStream_t s = as_stream(stream);
  for (int it = 0; it < n_iter; ++it) {
    const bool prior = prior_on(st);
    if (prior && st->iterations == 0) {
      const int rc = launch_tac_eval(d.kin, V, d.params, d.F, nullptr, s);
      if (rc) return rc;
    }
    if (prior && st->use_graph) {
      if (!st->exec) {
        const int rc = build_graph(st);
        if (rc) return rc;
      }
      KCS_CUDA(cudaGraphLaunch(st->exec, s));
    } else {
      const int rc = issue_iteration(st, prior, stream);
      if (rc) return rc;
    }
    st->iterations += 1;
  }
  return KCS_OK;
}

int kcs_icm_iterate_host(kcs_study_t* st, int n_iter, const void* counts_host,
                         float* params_host, size_t params_host_stride, void* stream) {
  clear_error();
  KCS_REQUIRE(st, "study is NULL");
  KCS_REQUIRE(n_iter >= 0, "n_iter < 0");
  const kcs_study_desc_t& d = st->d;
  const kcs_geometry* g = d.geom;
  const long long V = (long long)g->nz * g->ny * g->nx;
  const size_t counts_bytes = (size_t)g->nz * g->A * g->B * d.n_frames *
                              (d.counts_type == KCS_U16 ? 2 : 4);
  const size_t maps_bytes = sizeof(float) * 4 * (size_t)V;
  KCS_REQUIRE(params_host_stride == 0 || params_host_stride >= (size_t)4 * V,
              "params_host_stride %zu is neither 0 nor >= 4 x voxels", params_host_stride);
  if (n_iter == 0) return KCS_OK;
  if (!st->copy) {
    KCS_CUDA(cudaStreamCreateWithFlags(&st->copy, cudaStreamNonBlocking));
    for (auto& e : st->ev) KCS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  enum { OSL_DONE = 0, COUNTS_IN = 1, FIT_DONE = 2, MAPS_OUT = 3 };
  cudaStream_t s = as_stream(stream), c = st->copy;
  // everything already on the caller's stream (which may read the counts or
  // the maps) precedes the first copy
  KCS_CUDA(cudaEventRecord(st->ev[FIT_DONE], s));
  KCS_CUDA(cudaStreamWaitEvent(c, st->ev[FIT_DONE], 0));
  // The first upload goes subset by subset when the rows of a subset are
  // every S-th sinogram row of the volume (A a multiple of S, or one plane):
  // one strided copy each, and the first OSL pass starts on subset 0 while the
  // later subsets' rows are still arriving.  Later uploads overlap the fit.
  const size_t row_bytes = (size_t)g->B * d.n_frames * (d.counts_type == KCS_U16 ? 2 : 4);
  const bool by_subset = counts_host && g->S > 1 && (g->A % g->S == 0 || g->nz == 1);
  if (by_subset) {
    if (st->ev_sub.size() != (size_t)g->S) {
      st->ev_sub.assign(g->S, nullptr);
      for (auto& e : st->ev_sub) KCS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    for (int k = 0; k < g->S; ++k) {
      const size_t rows = g->A % g->S == 0 ? (size_t)g->nz * (g->A / g->S)
                                           : (size_t)subset_count(g, k);
      KCS_CUDA(cudaMemcpy2DAsync(static_cast<char*>(const_cast<void*>(d.counts)) + k * row_bytes,
                                 g->S * row_bytes,
                                 static_cast<const char*>(counts_host) + k * row_bytes,
                                 g->S * row_bytes, row_bytes, rows, cudaMemcpyHostToDevice, c));
      KCS_CUDA(cudaEventRecord(st->ev_sub[k], c));
    }
  } else if (counts_host) {
    KCS_CUDA(cudaMemcpyAsync(const_cast<void*>(d.counts), counts_host, counts_bytes,
                             cudaMemcpyHostToDevice, c));
  }
  KCS_CUDA(cudaEventRecord(st->ev[COUNTS_IN], c));
  KCS_CUDA(cudaEventRecord(st->ev[MAPS_OUT], c));
  for (int it = 0; it < n_iter; ++it) {
    const bool prior = prior_on(st);
    const bool sub_wait = by_subset && it == 0;
    if (!sub_wait) KCS_CUDA(cudaStreamWaitEvent(s, st->ev[COUNTS_IN], 0));   // this iteration's counts
    if (prior && st->iterations == 0) {
      const int rc = launch_tac_eval(d.kin, V, d.params, d.F, nullptr, s);
      if (rc) return rc;
    }
    int rc = issue_osl_pass(st, prior, s, sub_wait ? st->ev_sub.data() : nullptr);
    if (rc) return rc;
    // the next iteration's counts arrive while this one fits the maps (the
    // fit does not read the counts)
    KCS_CUDA(cudaEventRecord(st->ev[OSL_DONE], s));
    if (counts_host && it + 1 < n_iter) {
      KCS_CUDA(cudaStreamWaitEvent(c, st->ev[OSL_DONE], 0));
      KCS_CUDA(cudaMemcpyAsync(const_cast<void*>(d.counts), counts_host, counts_bytes,
                               cudaMemcpyHostToDevice, c));
      KCS_CUDA(cudaEventRecord(st->ev[COUNTS_IN], c));
    }
    // the previous iteration's maps have left before the fit overwrites them
    KCS_CUDA(cudaStreamWaitEvent(s, st->ev[MAPS_OUT], 0));
    rc = issue_fit(st, s);
    if (rc) return rc;
    st->iterations += 1;
    // this iteration's maps leave during the next OSL pass (which does not
    // touch them)
    if (params_host) {
      KCS_CUDA(cudaEventRecord(st->ev[FIT_DONE], s));
      KCS_CUDA(cudaStreamWaitEvent(c, st->ev[FIT_DONE], 0));
      KCS_CUDA(cudaMemcpyAsync(params_host + (size_t)it * params_host_stride, d.params,
                               maps_bytes, cudaMemcpyDeviceToHost, c));
      KCS_CUDA(cudaEventRecord(st->ev[MAPS_OUT], c));
    }
  }
  // the caller's stream completes with the last copy
  KCS_CUDA(cudaStreamWaitEvent(s, st->ev[MAPS_OUT], 0));
  return KCS_OK;
}

}  // extern "C"
