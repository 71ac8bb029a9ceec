// Internal interface of the batched ensemble step (pic_capi.cu): every run's step in one launch per kernel
// class, optionally replayed from a CUDA graph. Used by pic_ensemble.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/pic.h"

namespace picgb {

struct Batch {
  virtual ~Batch() {}
  virtual int step(int nsteps) = 0;
  virtual void use_graphs(bool on) = 0;
  virtual int64_t launches() const = 0;
};

// NULL (and *why) when the runs cannot share the batched kernels: the runs must be 2D contexts of one
// precision, shape order, solver family, filter and particle layout, loaded with plasma, without a test
// beam, lab samples or moving window, created on the stream s.
Batch* make_batch(pic_ctx* const* runs, int n, cudaStream_t s, std::string* why);

}  // namespace picgb
