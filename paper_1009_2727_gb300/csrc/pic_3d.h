// Internal interface of the 3D path (x, y, z) and of the 1D path (z): one object
// per context created with pic_config.dim == 3 or 1. The C entry points of
// pic_capi.cu forward to it.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/pic.h"

namespace picgb {

struct Sim3Api {
  virtual ~Sim3Api() {}
  virtual int load_plasma(const pic_plasma* p) = 0;
  virtual int set_laser(const pic_laser* l) = 0;
  virtual int run(int nsteps) = 0;
  virtual int sync() = 0;
  virtual int btd_set(const pic_btd_req* r) = 0;
  virtual int btd_get(pic_btd_out* o) = 0;
  virtual int get_field(int comp, double* dst, int on_device) = 0;
  virtual int set_field(int comp, const double* src) = 0;
  // any of x, y, z, ... may be NULL; with x == y == z == NULL only *count is set
  virtual int get_particles(int species, double* x, double* y, double* z, double* ux, double* uy, double* uz,
                            double* w, uint32_t* id, int32_t* flags, int64_t* count) = 0;
  virtual int stats(pic_stats* o) = 0;
  virtual int64_t launches() const = 0;
  virtual int kernel_timing(int enable, int which, double* ms_total, int64_t* n) = 0;
  // the frozen test beam's self-field added to the fields (3D only)
  virtual int beam_self_field() { return PIC_EINVAL; }
  virtual int status() const = 0;
  virtual const std::string& error() const = 0;
};

// Validates the 3D configuration and allocates the fields; on failure returns
// NULL and sets *status (and *err).
Sim3Api* make_sim3(const pic_config* cfg, pic_alloc_fn alloc, pic_free_fn free_fn, void* user, cudaStream_t s,
                   int* status, std::string* err);

// The same for the 1D configuration (pic_config.dim == 1).
Sim3Api* make_sim1(const pic_config* cfg, pic_alloc_fn alloc, pic_free_fn free_fn, void* user, cudaStream_t s,
                   int* status, std::string* err);

}  // namespace picgb
