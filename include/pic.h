/*
 * pic.h — C ABI of the GB300-native boosted-frame electromagnetic PIC step.
 *
 * The library advances a 2-1/2D (x,z; all six field components, three momentum
 * components, fields independent of y) or a 3D (x,y,z) laser-wakefield
 * simulation in a Lorentz boosted frame, following J.-L. Vay, C.G.R. Geddes, E. Cormier-Michel,
 * D.P. Grote, "Modeling laser wakefield accelerators in a Lorentz boosted
 * frame" (arXiv:1009.2727). Every step runs in the library's CUDA kernels
 * (sm_103a) on one GPU and one caller-supplied CUDA stream.
 *
 * Conventions
 *  - SI units. Lab-frame physical inputs (densities, laser, beam, stations) are
 *    transformed by the library.
 *  - Every function returns a pic_status (0 = PIC_OK, negative = error). Errors
 *    are sticky per context; pic_last_error() returns a text description.
 *  - Device memory is owned by the library and obtained only through the
 *    allocator callback given to pic_init (or cudaMalloc when it is NULL); it is
 *    released by pic_free. Caller buffers are never retained after a call.
 *  - A context is used from one host thread at a time; all device work is
 *    enqueued on the context's stream. pic_step is asynchronous.
 *  - Grid arrays are (nx+1) x (nz+1), row-major with z fastest: element (i,k)
 *    is at i*(nz+1)+k in every buffer this ABI copies out. Each component sits
 *    at its own Yee position: Ex (i+1/2,k), Ey (i,k), Ez (i,k+1/2),
 *    Bx (i,k+1/2), By (i+1/2,k+1/2), Bz (i+1/2,k); J like E.
 *  - 3D (pic_config.dim = 3): arrays are (nx+1) x (ny+1) x (nz+1), element
 *    (i,j,k) at (i*(ny+1)+j)*(nz+1)+k; Ex (i+1/2,j,k), Ey (i,j+1/2,k),
 *    Ez (i,j,k+1/2), Bx (i,j+1/2,k+1/2), By (i+1/2,j,k+1/2), Bz (i+1/2,j+1/2,k).
 *    3D contexts have no moving window, autotuner or pic_get_rho_noalloc;
 *    the laser antenna is at rest (beta_s = 0).
 *  - 1D (pic_config.dim = 1; App. I): fields and positions depend on z only,
 *    arrays are nz+1 values; Ex, Ey, Bz at k, Ez, Bx, By at k+1/2; nx, dx,
 *    the solver coefficients (the 1D operator is Yee's), ppc_x and the laser's
 *    w0 and x_center are ignored; the laser is a plane wave from a current
 *    sheet at rest; weights and the field energy are per unit transverse area;
 *    pic_get_particles returns the electrons (x = 0; the ions are a column
 *    current); the moving window runs in the lab frame (gamma_boost = 1);
 *    no test beam, lab-frame samples, autotuner or pic_get_rho_noalloc.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_API_VERSION 1

typedef enum {
  PIC_OK = 0,
  PIC_EINVAL = -1,     /* bad argument or configuration */
  PIC_ENOMEM = -2,     /* the allocator returned NULL */
  PIC_ECFL = -3,       /* dt above the stability limit (Eq. cfl with the Friedman factor) */
  PIC_EOVERFLOW = -4,  /* particle or lab-sample capacity exceeded */
  PIC_ECUDA = -5,      /* a CUDA runtime call failed */
  PIC_ETIMEOUT = -6,   /* a bounded device wait gave up */
  PIC_ENAN = -7,       /* a non-finite value was detected */
  PIC_ESTATE = -8      /* call out of order (e.g. pic_step before pic_load_plasma when required) */
} pic_status;

enum { PIC_FP64 = 0, PIC_MIXED = 1 };              /* pic_config.precision */
enum { PIC_EX = 0, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_JX, PIC_JY, PIC_JZ, PIC_RHO };
enum { PIC_ELECTRONS = 0, PIC_BEAM = 2 };            /* pic_get_particles species */

typedef struct pic_ctx pic_ctx;                      /* opaque, owned by the library */

/* Device allocator: returns a device pointer of at least `bytes` usable on
 * `stream`, or NULL. Called only inside pic_init/pic_load_plasma/
 * pic_boosted_to_lab_diag (never inside pic_step unless particle capacity must
 * grow). `user` is passed through. */
typedef void* (*pic_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*pic_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Numerical configuration. struct_size must be sizeof(pic_config) and version
 * PIC_API_VERSION. */
typedef struct {
  uint32_t struct_size, version;
  int32_t dim;            /* 2 (x,z), 3 (x,y,z) or 1 (z) */
  int32_t nx, nz;         /* cells along x and z; the PML occupies pml_cells on each side */
  double dz_lab;          /* lab longitudinal cell [m]; the computational cell is (1+beta) gamma dz_lab (Sec. 5.1.1) */
  double dx;              /* transverse cell [m] */
  double gamma_boost;     /* Lorentz factor of the computational frame (1 = lab) */
  double courant;         /* dt = courant * dt_CFL when dt <= 0 */
  double dt;              /* explicit time step [s], or <= 0 */
  double ck_alpha, ck_beta, ck_gamma; /* tunable-solver coefficients (Table CKcoefs), alpha+4beta+4gamma = 1 */
  double theta;           /* Friedman damping 0..1 (Eq. Faraday_Friedman) */
  int32_t pml_cells;      /* split-field PML thickness (App. II); 0 = PEC walls */
  double pml_sigma_max;   /* sigma_m in units of c/delta (paper: 4) */
  double pml_delta;       /* Delta in cells (paper: 5) */
  double pml_power;       /* profile exponent n (paper: 2) */
  int32_t pml_xi_exp;     /* 1: xi = exp(-sigma dt); 0: (1 - sigma dt/2)/(1 + sigma dt/2) */
  int32_t filter_passes;  /* bilinear passes per axis (Eq. 3ptfilter, alpha = 1/2); passes plus the
                             compensation pass <= 16 and the halo (that count) x (stride, or the sum of
                             filter_stride_set) <= 40, else PIC_EINVAL */
  int32_t filter_stride;  /* stride s (Eq. 3ptfilter_stride) */
  int32_t filter_compensate; /* 1: one extra pass with alpha_c = n/2 + 1 */
  int32_t filter_J;       /* filter the deposited current */
  int32_t filter_gather;  /* filter the fields used by the gather */
  int32_t shape_order;    /* 1 or 3 */
  int32_t particle_guard; /* cells between the PML and the particle domain; < 0 = default */
  int32_t precision;      /* PIC_FP64 or PIC_MIXED (FP32 fields/momenta, FP64 positions and PML coefficients) */
  int32_t moving_window;  /* 1: the grid follows the wake at window_beta c */
  double window_beta;
  int32_t tile_x, tile_z; /* particle tile in cells (x, z); 0 = default 8 x 32; at most 1024 cells */
  int32_t sort_every;     /* steps between particle sorts; 0 = default */
  int32_t ny;             /* 3D: cells along y (the PML occupies pml_cells on each side) */
  int32_t gather_scheme;  /* 0: 'energy conserving' gather from the Yee locations (Sec. 5, the paper's
                             default); 1: 'momentum conserving': the gather copies are first
                             interpolated to the nodes (mean of the two, or four, nearest staggered
                             values), then gathered with node-centred shapes; else PIC_EINVAL */
  double dy;              /* 3D: transverse cell along y [m] */
  int32_t filter_stride_set[4]; /* wide-band filter (Sec. 4.1): along each axis the passes (and the
                                   compensation pass) are applied at each of these strides in turn, e.g.
                                   {1, 2, 3, 0}; 0-terminated, all zero = the single filter_stride;
                                   a negative entry or a stride after a 0 is PIC_EINVAL */
} pic_config;

/* Cold plasma fixed in the lab (Sec. 3.1.1), on a regular lattice, entering the
 * boosted box through the plane at the +z edge of the particle domain. */
typedef struct {
  uint32_t struct_size, version;
  double n0;              /* lab electron density of the plateau [m^-3] */
  double z_start_lab;     /* lab position where the linear entrance ramp starts [m] */
  double ramp_lab;        /* lab length of the linear ramp [m] */
  double length_lab;      /* lab length of the plateau [m]; <= 0 = unbounded */
  int32_t ppc_x, ppc_z;   /* macro-particles per cell along x and z */
  int32_t ions;           /* 1: neutralising ions fixed in the lab, same lattice */
  /* optional test beam (Sec. 3.1.1): beam_n lab-frame particles given at lab
   * time beam_t_lab, injected through the lab plane z = beam_z_plane_lab.
   * Host pointers, read during the call only; u = gamma v [m/s]. */
  int64_t beam_n;
  const double *beam_x, *beam_z, *beam_ux, *beam_uy, *beam_uz;
  double beam_t_lab, beam_z_plane_lab;
  const double* beam_y;   /* 3D: beam y positions (host, beam_n values) */
  int32_t ppc_y;          /* 3D: macro-particles per cell along y (0 = 1) */
  int32_t beam_self;      /* 2D: 1 = self-consistent beam (Sec. 3.1.1): its frozen particles inside the
                             particle domain deposit the current of their move at the mean velocity and
                             its active particles deposit like the plasma; needs beam_w. The caller sets
                             the beam's initial self-field (pic_set_field). 0 = test particles.
                             PIC_EINVAL when beam_w is NULL, and in 3D (1D takes no test beam at all) */
  const double* beam_w;   /* beam weights: macro-particle counts per unit length along y (host, beam_n
                             values; read only with beam_self) */
  int32_t reserved[2];
} pic_plasma;

/* Gaussian laser injected through a plane (Sec. 3.1.2). The lab waveform at the
 * antenna is E0 exp(-(x-x_center)^2/w0^2) exp(-(s-t_peak)^2/(2 sigma_t^2))
 * sin(omega (s - t_peak) + phase), sigma_t = tau_fwhm/(2 sqrt(ln 2)), y-polarised;
 * in 3D the transverse factor is exp(-((x-x_center)^2 + (y-y_center)^2)/w0^2) and
 * the current comes from dual particle arrays (one pair per transverse node of the
 * particle domain, the moving partner displaced along y, Esirkepov deposition). */
typedef struct {
  uint32_t struct_size, version;
  double lambda0, a0, w0, tau_fwhm, t_peak, x_center, phase;
  double z_antenna;       /* antenna position in the computational frame at t' = 0 [m]; the antenna
                             emits only while it lies inside the particle domain (past the PML and the
                             particle guard, whose default width grows with the filter's halo) */
  double beta_s;          /* antenna-plane velocity / c in the computational frame */
  double y_center;        /* 3D: laser axis position along y [m] */
  int32_t reserved[6];
} pic_laser;

/* Back-transformed diagnostics (Sec. 3.2): n_rows lab samples (z_lab[r], t_lab[r])
 * each covering all nx+1 transverse positions and the six lab-frame components. */
typedef struct {
  uint32_t struct_size, version;
  int64_t n_rows;
  const double* z_lab;    /* host pointers, copied during the call */
  const double* t_lab;
} pic_btd_req;

typedef struct {
  uint32_t struct_size, version;
  void* data;             /* n_rows * 6 * (nx+1) values of the context precision's real type
                             (double for PIC_FP64, float for PIC_MIXED), layout [row][component][i]
                             (3D: [row][component][i][j]); NULL: only the counts are returned */
  int32_t* done;          /* n_rows * 2 flags: E part complete, B part complete (may be NULL) */
  int32_t on_device;      /* 1: data/done are device pointers, 0: host pointers */
  int64_t n_rows_filled;  /* out: rows with both parts complete */
} pic_btd_out;

typedef struct {
  uint32_t struct_size, version;
  int64_t step;
  double t;               /* computational-frame time [s] */
  double dt, dx, dz, gamma, beta;
  int64_t n_electrons;    /* live plasma electrons */
  int64_t n_beam_active;
  double beam_gamma_lab;  /* mean lab-frame Lorentz factor of the active test beam */
  double beam_spread;     /* rms(gamma_lab)/mean */
  double field_energy;    /* per unit length along y [J/m] in 2D; [J] in 3D */
  int32_t gx_lo, gx_hi, gz_lo, gz_hi; /* particle domain in cells */
  int64_t sorts, overflow_chunks;     /* runtime counters */
  double z0;              /* grid origin (moving window) [m] */
  double trap_gamma_lab;  /* in: a threshold > 0 to use, else 0; out: the threshold used, by default
                             2 gamma_w, gamma_w = omega_laser / omega_p (0: no laser or plasma) */
  double trapped_charge;  /* charge of the plasma electrons whose lab-frame gamma exceeds it, per unit
                             length along y [C/m] */
} pic_stats;

/* Create a context: validates cfg (coefficient normalisation, shape order,
 * dt against the stability limit -> PIC_ECFL), derives the boosted cell and
 * time step, allocates and zeroes the fields. The solver coefficients and the
 * stability limit follow Sec. 4.2.1 (Table CKcoefs, Eq. cfl) and Sec. 4.3 (the
 * Friedman factor); the boosted cell follows Sec. 5.1.1; the PML App. II. cuda_stream is a cudaStream_t
 * (NULL = the legacy default stream). On error *out is NULL. */
int pic_init(const pic_config* cfg, pic_alloc_fn alloc, pic_free_fn free_fn, void* alloc_user,
             void* cuda_stream, pic_ctx** out);

/* Load the plasma (rows inside the particle domain at t' = 0) and, optionally,
 * the test beam (both as injected through a plane, Sec. 3.1.1). May be called
 * once, before the first pic_step. */
int pic_load_plasma(pic_ctx* ctx, const pic_plasma* plasma);

/* Register the laser antenna (Sec. 3.1.2); its current is deposited inside every pic_step. */
int pic_inject_laser(pic_ctx* ctx, const pic_laser* laser);

/* Advance nsteps steps (asynchronous on the context stream). One step: Faraday
 * with the tunable operator and Friedman damping (Eq. Faraday, Eq.
 * Faraday_Friedman) and the PML (App. II); the field gather and Boris push;
 * Esirkepov deposition (Sec. 4.2.2); the antenna; the filter (Sec. 4.1) of the
 * current and of the gathered fields; Ampere (Eq. Ampere); inflow, removal and
 * the moving window (Sec. 3.1.1, Sec. 2). Returns a host-side status;
 * device-side errors are reported by pic_sync. */
int pic_step(pic_ctx* ctx, int nsteps);

/* Wait for the stream and return the sticky device status. */
int pic_sync(pic_ctx* ctx);

/* Lab-frame stations/snapshots (Sec. 3.2). With req != NULL and out == NULL: register the
 * sample rows (replacing any previous request) and zero their buffers; they are
 * filled while stepping. With req == NULL and out != NULL: copy the rows out
 * (synchronises the stream). */
int pic_boosted_to_lab_diag(pic_ctx* ctx, const pic_btd_req* req, pic_btd_out* out);

/* Release all device memory and the context. NULL is accepted. */
int pic_free(pic_ctx* ctx);

/* Accessors (synchronise the stream). */
/* Copy one grid component (PIC_EX..PIC_JZ, or PIC_RHO = charge density of
 * electrons and ions at the current positions) into dst: (nx+1)*(nz+1) values
 * of type double (always converted to double). on_device selects dst memory. */
int pic_get_field(pic_ctx* ctx, int comp, double* dst, int on_device);
/* Overwrite one of the six E/B components from a host array of doubles (tests). */
int pic_set_field(pic_ctx* ctx, int comp, const double* src);
/* Copy the live particles of one species to host arrays of capacity *count
 * (doubles; id as uint32). On return *count is the number of live particles.
 * flags (may be NULL): bit0 alive, bit1 active (test beam). Pass x == NULL to
 * query the count only. */
int pic_get_particles(pic_ctx* ctx, int species, double* x, double* z, double* ux, double* uy,
                      double* uz, double* w, uint32_t* id, int32_t* flags, int64_t* count);
int pic_get_stats(pic_ctx* ctx, pic_stats* out);
/* 3D contexts: the y positions [m] of the particles pic_get_particles returns,
 * in the same order (*count as there); PIC_EINVAL for 2D contexts. */
int pic_get_particles_y(pic_ctx* ctx, int species, double* y, int64_t* count);
const char* pic_last_error(pic_ctx* ctx);

/* Self-field of the frozen test beam, solved on the device and added to the
 * fields (Sec. 3.1.1: the fields at the injection plane must be consistent with
 * the beam, whose charge the frozen and the active particles deposit; reading
 * PR-27). The frozen particles inside the particle domain are a charge moving
 * rigidly at the beam's mean velocity v along z: the potential solves
 * d2phi/dx2 + d2phi/dz2 / gamma_v^2 = -rho/eps0 with phi = 0 on the PEC walls,
 * in the Yee mesh's second differences (so that the discrete Gauss law holds
 * exactly), by sine transforms (DST-I) along both axes; E_x = -dphi/dx and
 * E_z = -dphi/dz / gamma_v^2 are added to E at the current time, B_y = v E_x / c^2
 * from the positions half a step earlier to B (B^{n-1/2}). Call it once, after
 * pic_load_plasma and before the first pic_step, for a beam loaded with
 * pic_plasma.beam_self = 1. 2D contexts only (PIC_EINVAL otherwise);
 * PIC_ESTATE without a self-consistent beam. Scratch of two grid-sized FP64
 * arrays comes from the allocator callback and is released before it returns;
 * the call synchronises the context's stream. */
int pic_beam_self_field(pic_ctx* ctx);

/* Largest nz accepted by pic_get_rho_noalloc (size of its static scratch). */
#define PIC_NOALLOC_MAX_NZ 16384

/* Charge density without any device allocation. Same result as
 * pic_get_field(ctx, PIC_RHO, dst_device, 1), for callers that must not
 * allocate device memory once their run is set up: for example an application
 * whose device memory is entirely owned by its own pool allocator, or a
 * real-time loop that cannot afford the latency and implicit device
 * synchronisation of cudaMalloc/cudaFree. (The paper has no counterpart: this
 * is a service of the library, not part of the method.)
 *  - dst_device: caller-owned device buffer of (nx+1)*(nz+1) doubles, written in
 *    the layout of pic_get_field. It is zeroed and filled on the context's
 *    stream; the call returns without waiting (pic_sync or a stream
 *    synchronisation makes the result visible to the host).
 *  - 2D contexts only: 1D and 3D contexts return PIC_EINVAL.
 *  - The ion row density is staged in a file-scope static device array of
 *    PIC_NOALLOC_MAX_NZ+1 doubles (128 KiB) that every GPU loading the library
 *    keeps until the process exits. Every call looks up that array's device
 *    address (cudaGetSymbolAddress, with the caller's device current; the
 *    lookup allocates nothing). The first call on a device may load the
 *    library's device code there: make it before any stream capture.
 *  - All calls share the array and it keeps the last call's contents; calls
 *    whose work overlaps on the GPU (several contexts or streams at once) race.
 *  - nz > PIC_NOALLOC_MAX_NZ is rejected with PIC_EINVAL (pic_last_error says
 *    why). No cudaMalloc, cudaFree or allocator callback is used. */
int pic_get_rho_noalloc(pic_ctx* ctx, double* dst_device);

/* Number of kernel launches enqueued so far by this context (bench accounting). */
int64_t pic_kernel_launches(pic_ctx* ctx);

/* Measured FP32 arithmetic peak of the current device, in TFLOP/s: the best of
 * five launches of a kernel whose threads run eight independent FMA chains
 * over every SM (two FLOPs per FMA lane), once with scalar FMAs and once with
 * the packed two-lane FMA of sm_100 and later. The denominator of the push
 * kernel's arithmetic roofline (the paper measures no GPU; this is a
 * measurement service of the library). Allocates one small scratch buffer
 * with cudaMalloc and frees it; synchronises the device. Returns PIC_EINVAL
 * for null outputs, PIC_ENOMEM or PIC_ECUDA on CUDA failures. */
int pic_measure_fp32_peak(double* scalar_tflops, double* packed_tflops);

/* Record CUDA events around the launches of the named kernel class in the next
 * pic_step calls and return their summed duration in ms (0 = particle kernel,
 * 1 = field kernels). Used by the benchmark for the per-kernel roofline. */
int pic_kernel_timing(pic_ctx* ctx, int enable, int which, double* ms_total, int64_t* launches);

/* ---- Autotuner of the particle layout (no counterpart in the paper) ----
 * Picks the particle tile (tile_x, tile_z) from {8, 16, 32}^2 at a cadence of 32,
 * then the sort cadence from {8, 16, 32, 64, 128} for that tile, by timing `steps`
 * steps (after 4 warm-up steps; a cadence trial runs at least two sort periods;
 * each tile is timed twice and the faster time is recorded, after one untimed
 * trial that brings the GPU to its clocks) of contexts built from cfg, plasma and
 * laser (laser may be NULL) through
 * pic_init/pic_load_plasma/pic_inject_laser with the given allocator and stream.
 * The result is cached per (nx, nz, ppc_x, ppc_z, shape order, precision,
 * gamma_boost, warm-up and timed steps) for the life of the process; a cached answer comes back without
 * timing and with cached = 1. out->struct_size must be set by the caller.
 * Returns PIC_EINVAL for bad arguments, PIC_ECUDA when no trial ran. */
#define PIC_TUNE_MAX_TRIALS 16
typedef struct pic_tune_result {
  uint32_t struct_size;
  uint32_t version;
  int32_t tile_x, tile_z, sort_every;   /* the chosen layout */
  double ms_per_step;                   /* its time per step in the trials */
  int32_t n_trials;
  int32_t trial_tile_x[PIC_TUNE_MAX_TRIALS];
  int32_t trial_tile_z[PIC_TUNE_MAX_TRIALS];
  int32_t trial_sort_every[PIC_TUNE_MAX_TRIALS];
  double trial_ms[PIC_TUNE_MAX_TRIALS]; /* < 0: the trial failed */
  int32_t cached;
} pic_tune_result;

int pic_autotune(const pic_config* cfg, const pic_plasma* plasma, const pic_laser* laser, int steps,
                 pic_alloc_fn alloc, pic_free_fn free_fn, void* alloc_user, void* cuda_stream,
                 pic_tune_result* out);
/* The same with the window of the run that the trials time: `warm` untimed steps (instead of 4), then
 * `steps` timed steps; a layout that is best while the plasma is still cold need not be best once the
 * laser has reached it, so a caller that times a later window tunes on that window. The cache key
 * includes warm and steps. Errors as pic_autotune (warm < 0: PIC_EINVAL). */
int pic_autotune_window(const pic_config* cfg, const pic_plasma* plasma, const pic_laser* laser, int warm,
                        int steps, pic_alloc_fn alloc, pic_free_fn free_fn, void* alloc_user, void* cuda_stream,
                        pic_tune_result* out);

/* ---- Ensemble of independent runs (no counterpart in the paper) ----
 * n runs of uneven size (each its own pic_config, pic_plasma and pic_laser;
 * lasers may be NULL, and a laser with lambda0 <= 0 means none) advanced together.
 * Every run is an ordinary context created and owned by the ensemble.
 *  - Batched mode (2D runs with plasma, the Yee-located gather, no lab samples,
 *    no moving window, one precision, shape order, solver family, damping, filter
 *    and particle layout; at most 512 runs; a test beam rides along): all runs
 *    share one non-blocking stream and an ensemble step is one launch per kernel
 *    class over all runs (Faraday, gather filter, push, its global pass, test
 *    beams, antenna, ion current, Ampere, inflow, counts; the runs' sorts every
 *    sort_every steps), the per-run
 *    arguments of the step in one block of device memory filled from the same
 *    host decisions as pic_step. From the third step on, each step replays a
 *    CUDA graph of those launches (pic_ensemble_use_graphs(ens, 0) launches them
 *    directly instead). A run that gains lab samples afterwards makes
 *    pic_ensemble_step fail with PIC_ESTATE.
 *  - Otherwise every run has its own non-blocking stream and pic_ensemble_step
 *    enqueues one step of every run before the next, so that they run
 *    concurrently.
 * The runs start after the work already on cuda_stream, and cuda_stream waits
 * for all of them when pic_ensemble_step returns (pass NULL to skip both).
 * pic_ensemble_member gives a run's context for the accessors (pic_get_field,
 * pic_get_stats, ...); it stays owned by the ensemble. Errors: PIC_EINVAL for bad
 * arguments, else the first failing call's status; pic_ensemble_sync returns the
 * first run's error. */
typedef struct pic_ens pic_ens;
int pic_ensemble_create(int n, const pic_config* cfgs, const pic_plasma* plasmas, const pic_laser* lasers,
                        pic_alloc_fn alloc, pic_free_fn free_fn, void* alloc_user, void* cuda_stream,
                        pic_ens** out);
int pic_ensemble_step(pic_ens* ens, int nsteps);
int pic_ensemble_sync(pic_ens* ens);
int pic_ensemble_size(pic_ens* ens);
/* 1 when the ensemble steps in batched mode, else 0 */
int pic_ensemble_batched(pic_ens* ens);
/* batched mode: replay each step from a CUDA graph (1, the default) or launch directly (0) */
int pic_ensemble_use_graphs(pic_ens* ens, int enable);
/* kernel launches enqueued so far by the ensemble's steps (bench accounting) */
int64_t pic_ensemble_launches(pic_ens* ens);
pic_ctx* pic_ensemble_member(pic_ens* ens, int index);
int pic_ensemble_free(pic_ens* ens);
/* The particle tile and sort cadence for a whole ensemble: each candidate layout (tiles 8x32, 8x16, 16x16,
 * 16x32, 32x32, 8x8 at cadence 32; 8x32 at cadences 16 and 64) is given to every run, the ensemble is
 * created, stepped 4 times, then timed over `steps` ensemble steps on cuda_stream; out receives the
 * fastest layout, its ms per ensemble step and every trial (ms < 0 for a failed one). The runs' own
 * tile_x/tile_z/sort_every in cfgs are ignored. Errors: PIC_EINVAL, PIC_ECUDA (no candidate ran). */
int pic_ensemble_autotune(int n, const pic_config* cfgs, const pic_plasma* plasmas, const pic_laser* lasers,
                          int steps, pic_alloc_fn alloc, pic_free_fn free_fn, void* alloc_user, void* cuda_stream,
                          pic_tune_result* out);

/* ---- Multilayer perceptron for the stage surrogate (no counterpart in the paper) ----
 * widths[0] -> widths[1] -> ... -> widths[n_layers]; GELU (exact, erf form) after every layer but the
 * last. Parameters: per layer l = 1..n_layers the weight W_l (widths[l] x widths[l-1], row-major) then
 * the bias b_l (widths[l]); FP32 master copies updated by AdamW, BF16 copies used by every product;
 * activations stored in BF16; products accumulate in FP32. Initial weights are uniform in
 * +-sqrt(6 / fan_in) (half that for the last layer) from a splitmix64 sequence seeded by seed; biases 0.
 * Device pointers: x (n x widths[0]), t and y (n x widths[n_layers]), FP32 row-major, on the MLP's
 * stream. pic_mlp_grad returns the mean squared error of the outputs against t and its gradient with
 * respect to all parameters (host buffers, pic_mlp_param_count floats). pic_mlp_train runs `epochs`
 * passes of minibatches of `batch` rows in a splitmix64-shuffled order (the remainder of each pass is
 * skipped) with AdamW (beta 0.9/0.999, eps 1e-8, decoupled weight decay); loss_curve (host, epochs
 * floats, may be NULL) receives each pass's mean batch loss. Errors: PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA. */
typedef struct pic_mlp pic_mlp;
int pic_mlp_create(int n_layers, const int* widths, uint64_t seed, pic_alloc_fn alloc, pic_free_fn free_fn,
                   void* alloc_user, void* cuda_stream, pic_mlp** out);
int pic_mlp_free(pic_mlp* mlp);
int64_t pic_mlp_param_count(pic_mlp* mlp);
int pic_mlp_get_params(pic_mlp* mlp, float* dst_host);
int pic_mlp_set_params(pic_mlp* mlp, const float* src_host);
int pic_mlp_infer(pic_mlp* mlp, const float* x_device, int64_t n, float* y_device);
/* pic_mlp_infer is asynchronous. With every padded width (multiple of 16) <= 256 and at most 16 layers it
 * runs one fused tcgen05 kernel (128 rows per CTA, BF16 operands in shared memory, FP32 accumulators in
 * tensor memory, weights rebuilt into packed images after any parameter change); otherwise, or after
 * pic_mlp_use_tensor_cores(mlp, 0), the tiled CUDA-core GEMMs (PIC_EINVAL when enabling is impossible).
 * pic_mlp_status synchronises the stream and returns PIC_ETIMEOUT if a bounded tensor-core wait gave up. */
int pic_mlp_use_tensor_cores(pic_mlp* mlp, int enable);
int pic_mlp_status(pic_mlp* mlp);
int pic_mlp_grad(pic_mlp* mlp, const float* x_device, const float* t_device, int n, float* loss_host,
                 float* grad_host);
int pic_mlp_train(pic_mlp* mlp, const float* x_device, const float* t_device, int n, int epochs, int batch,
                  float lr, float weight_decay, uint64_t seed, float* loss_curve_host);
/* pic_mlp_train with epochs > 1 captures one epoch's launches (gather, forward, backward, AdamW per
 * minibatch; the epoch index and AdamW's bias corrections read on the device from a table the host fills
 * as the per-step launches would) in a CUDA graph on a private stream ordered after the MLP's stream,
 * and replays it once per epoch after uploading that epoch's order; the parameters come out bitwise the
 * same as from the direct launches. pic_mlp_use_graphs(mlp, 0) selects the direct launches on the MLP's
 * stream, as does a stream that is itself being captured. Errors: PIC_EINVAL (mlp NULL). */
int pic_mlp_use_graphs(pic_mlp* mlp, int enable);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
