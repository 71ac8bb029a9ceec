// Ensemble of independent runs (uneven grids, densities, boosts) advanced
// together: every run is an ordinary context on its own non-blocking stream,
// and a step of the ensemble enqueues one step of every run before waiting on
// any, so that the GPU executes the runs concurrently (small runs alone leave
// most SMs idle).
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "pic_batch.h"

struct pic_ens {
  std::vector<pic_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  cudaStream_t caller = nullptr;
  cudaEvent_t start = nullptr;
  std::vector<cudaEvent_t> done;
  // batched mode: every run on streams[0], one launch per kernel class per step (see pic_batch.h)
  std::unique_ptr<picgb::Batch> batch;
  std::string why_not_batched;
};

namespace {

// runs that the batched step may carry, judged from their inputs: 2D, the Yee-located gather, plasma, no
// moving window, one precision, shape order and particle layout (a test beam rides along)
bool batch_candidates(int n, const pic_config* cfgs, const pic_plasma* plasmas) {
  for (int i = 0; i < n; i++) {
    const pic_config& c = cfgs[i];
    if ((c.dim != 0 && c.dim != 2) || c.gather_scheme != 0 || c.moving_window) return false;
    if (!(plasmas[i].n0 > 0.0)) return false;
    if (c.precision != cfgs[0].precision || c.shape_order != cfgs[0].shape_order || c.tile_x != cfgs[0].tile_x ||
        c.tile_z != cfgs[0].tile_z || c.sort_every != cfgs[0].sort_every)
      return false;
  }
  return true;
}

void destroy(pic_ens* e) {
  e->batch.reset();
  for (pic_ctx* c : e->ctx) pic_free(c);
  for (cudaStream_t s : e->streams) cudaStreamDestroy(s);
  for (cudaEvent_t ev : e->done) cudaEventDestroy(ev);
  if (e->start) cudaEventDestroy(e->start);
  delete e;
}

}  // namespace

extern "C" {

int pic_ensemble_create(int n, const pic_config* cfgs, const pic_plasma* plasmas, const pic_laser* lasers,
                        pic_alloc_fn alloc, pic_free_fn free_fn, void* alloc_user, void* cuda_stream,
                        pic_ens** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (n < 1 || !cfgs || !plasmas) return PIC_EINVAL;
  pic_ens* e = new pic_ens();
  e->caller = (cudaStream_t)cuda_stream;
  if (cudaEventCreateWithFlags(&e->start, cudaEventDisableTiming) != cudaSuccess) {
    destroy(e);
    return PIC_ECUDA;
  }
  // runs the batched step can carry share one stream; otherwise each run gets its own
  const bool cand = batch_candidates(n, cfgs, plasmas);
  for (int i = 0; i < n; i++) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    if (!cand || i == 0) {
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        if (s) cudaStreamDestroy(s);
        destroy(e);
        return PIC_ECUDA;
      }
      e->streams.push_back(s);
      e->done.push_back(ev);
    } else {
      s = e->streams[0];
    }
    pic_ctx* c = nullptr;
    int r = pic_init(&cfgs[i], alloc, free_fn, alloc_user, s, &c);
    if (r != PIC_OK) {
      destroy(e);
      return r;
    }
    e->ctx.push_back(c);
    r = pic_load_plasma(c, &plasmas[i]);
    if (r == PIC_OK && lasers && lasers[i].lambda0 > 0.0) r = pic_inject_laser(c, &lasers[i]);
    if (r != PIC_OK) {
      destroy(e);
      return r;
    }
  }
  if (cand) {
    e->batch.reset(picgb::make_batch(e->ctx.data(), n, e->streams[0], &e->why_not_batched));
    // runs that the batched kernels cannot share after all step one after another on the common stream
  } else {
    e->why_not_batched = "runs outside the batched step (3D/1D, beam, window, node gather or mixed layouts)";
  }
  *out = e;
  return PIC_OK;
}

int pic_ensemble_step(pic_ens* e, int nsteps) {
  if (!e || nsteps < 0) return PIC_EINVAL;
  // the runs start after the work already on the caller's stream, and the caller's stream waits for all
  // of them at the end (also when it is the legacy default stream, handle 0: the runs' streams are
  // non-blocking and would not synchronise with it implicitly)
  cudaEventRecord(e->start, e->caller);
  for (cudaStream_t s : e->streams) cudaStreamWaitEvent(s, e->start, 0);
  if (e->batch) {
    const int r = e->batch->step(nsteps);
    if (r != PIC_OK) return r;
  } else {
    for (int k = 0; k < nsteps; k++)
      for (pic_ctx* c : e->ctx) {
        const int r = pic_step(c, 1);
        if (r != PIC_OK) return r;
      }
  }
  for (size_t i = 0; i < e->streams.size(); i++) {
    cudaEventRecord(e->done[i], e->streams[i]);
    cudaStreamWaitEvent(e->caller, e->done[i], 0);
  }
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_ensemble_sync(pic_ens* e) {
  if (!e) return PIC_EINVAL;
  int first = PIC_OK;
  for (pic_ctx* c : e->ctx) {
    const int r = pic_sync(c);
    if (r != PIC_OK && first == PIC_OK) first = r;
  }
  return first;
}

int pic_ensemble_size(pic_ens* e) { return e ? (int)e->ctx.size() : 0; }

int pic_ensemble_batched(pic_ens* e) { return e && e->batch ? 1 : 0; }

int pic_ensemble_use_graphs(pic_ens* e, int enable) {
  if (!e) return PIC_EINVAL;
  if (e->batch) e->batch->use_graphs(enable != 0);
  return PIC_OK;
}

int64_t pic_ensemble_launches(pic_ens* e) {
  if (!e) return 0;
  if (e->batch) return e->batch->launches();
  int64_t t = 0;
  for (pic_ctx* c : e->ctx) t += pic_kernel_launches(c);
  return t;
}

pic_ctx* pic_ensemble_member(pic_ens* e, int i) {
  if (!e || i < 0 || i >= (int)e->ctx.size()) return nullptr;
  return e->ctx[i];
}

// Layout of the whole ensemble: the particle tile and sort cadence shared by all runs, chosen by timing
// the ensemble itself (a layout that is fastest for one run alone on the GPU is not the fastest when the
// runs share it: small tiles multiply the chunk windows every run stages).
int pic_ensemble_autotune(int n, const pic_config* cfgs, const pic_plasma* plasmas, const pic_laser* lasers,
                          int steps, pic_alloc_fn alloc, pic_free_fn free_fn, void* alloc_user, void* cuda_stream,
                          pic_tune_result* out) {
  if (!out || out->struct_size != sizeof(pic_tune_result) || n < 1 || !cfgs || !plasmas || steps < 1)
    return PIC_EINVAL;
  static const int cand[][3] = {{8, 32, 32}, {8, 16, 32}, {16, 16, 32}, {16, 32, 32},
                                {32, 32, 32}, {8, 32, 16}, {8, 32, 64}, {8, 8, 32}};
  const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
  pic_tune_result r{};
  r.struct_size = sizeof(pic_tune_result);
  r.version = PIC_API_VERSION;
  double best = -1.0;
  std::vector<pic_config> c(cfgs, cfgs + n);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PIC_ECUDA;
  for (int q = 0; q < ncand; q++) {
    for (int i = 0; i < n; i++) {
      c[i].tile_x = cand[q][0];
      c[i].tile_z = cand[q][1];
      c[i].sort_every = cand[q][2];
    }
    pic_ens* e = nullptr;
    double ms = -1.0;
    if (pic_ensemble_create(n, c.data(), plasmas, lasers, alloc, free_fn, alloc_user, cuda_stream, &e) == PIC_OK &&
        pic_ensemble_step(e, 4) == PIC_OK && pic_ensemble_sync(e) == PIC_OK) {
      cudaEventRecord(e0, st);
      const int rr = pic_ensemble_step(e, steps);
      cudaEventRecord(e1, st);
      float t = 0.0f;
      if (rr == PIC_OK && pic_ensemble_sync(e) == PIC_OK && cudaEventSynchronize(e1) == cudaSuccess &&
          cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
        ms = (double)t / steps;
    }
    pic_ensemble_free(e);
    if (r.n_trials < PIC_TUNE_MAX_TRIALS) {
      const int i = r.n_trials++;
      r.trial_tile_x[i] = cand[q][0];
      r.trial_tile_z[i] = cand[q][1];
      r.trial_sort_every[i] = cand[q][2];
      r.trial_ms[i] = ms;
    }
    if (ms > 0.0 && (best < 0.0 || ms < best)) {
      best = ms;
      r.tile_x = cand[q][0];
      r.tile_z = cand[q][1];
      r.sort_every = cand[q][2];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0.0) return PIC_ECUDA;
  r.ms_per_step = best;
  *out = r;
  return PIC_OK;
}

int pic_ensemble_free(pic_ens* e) {
  if (!e) return PIC_OK;
  for (cudaStream_t s : e->streams) cudaStreamSynchronize(s);
  destroy(e);
  return PIC_OK;
}

}  // extern "C"
