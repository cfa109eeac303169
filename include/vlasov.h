/*
 * vlasov.h -- C ABI of libvlasov.so, a GB300 (sm_103a) solver for the one-dimensional Vlasov
 * equation with long-range mean-field forces, by the semi-Lagrangian Strang split of
 * T. M. Rocha Filho, arXiv:1206.3229 (Sec. 3):
 *
 *   step 1  f^(I)(x,p)    = f(x - p dt/2, p)            Eq. (step1)
 *   step 2  F^(I)(x)      = mean-field force of f^(I)   Eq. (step2), (meanforce)
 *   step 3  f^(II)(x,p)   = f^(I)(x, p - F^(I)(x) dt)   Eq. (step3)
 *   step 4  f(x,p,t+dt)   = f^(II)(x - p dt/2, p)       Eq. (step4)
 *
 * Every shift takes the cubic-spline value at the foot of the characteristic, Eqs. (splinegen,
 * splinecoeffs), with f'' from the eighth-order 9-point central difference, Eq. (findif).
 *
 * Storage (Sec. 3): f[j*Nx + i] with x (theta) contiguous, j the momentum row.  Nodes are
 * x_i = xmin + i*dx, dx = (xmax-xmin)/Nx and p_j = pmin + j*dp, dp = (pmax-pmin)/Np.
 *
 * Conventions for every entry point:
 *  - Return 0 (VLASOV_OK) or a negative VLASOV_E* code; no call aborts the process.  The text of
 *    the last error of the calling thread is returned by vlasov_last_error().
 *  - Host arrays are borrowed for the duration of the call and copied; device arrays named
 *    "dev_*" must be device memory of the current device, and stay owned by the caller.
 *  - One simulation handle must not be used by two threads at once; different handles are
 *    independent.  Work is enqueued on the handle's stream; calls documented as "syncs" wait for it.
 */
#ifndef VLASOV_H
#define VLASOV_H

#ifdef __cplusplus
extern "C" {
#endif

#define VLASOV_OK 0
#define VLASOV_EINVAL (-1)   /* bad argument: sizes, domain, dt, model, precision */
#define VLASOV_ENOMEM (-2)   /* device or host allocation failed */
#define VLASOV_ECUDA (-3)    /* a CUDA runtime/driver call failed (message has the CUDA text) */
#define VLASOV_ETIMEOUT (-4) /* a bounded device-side wait expired; results of that step are void */
#define VLASOV_ESTATE (-5)   /* call not valid in the handle's state (e.g. step before set_f) */
#define VLASOV_ERANGE (-6)   /* VLASOV_F64: |f| grew beyond the fixed-point range; results void */

/* Force models of Sec. 2.  FREE has F = 0 (free streaming; for tests). */
enum { VLASOV_HMF = 0, VLASOV_RING = 1, VLASOV_SHEET = 2, VLASOV_FREE = 3 };

/* Storage/arithmetic of f.
   F64: double storage.  The spline filter runs on integer and FP32 units (FP64 arithmetic is slow
        on this GPU): products of the high parts are exact int64 on a fixed-point grid of 2^-31 of a
        bound 2^Ef >= 4 max|f| (Ef from the last upload), residuals in FP32; error per sweep about
        2^-49 of 2^Ef, the size of FP64 rounding noise.  Needs |f| < 2^(Ef+1) (else VLASOV_ERANGE).
   F32: float storage and interpolation; displacements and all moment sums stay FP64-accurate.
   F64_NATIVE: double storage, IEEE FP64 filter arithmetic (reference; FP64-pipe bound).
   FX64: 64-bit fixed-point storage, f = X * 2^(Ef-62) with X int64 (same 8 bytes per cell; absolute
        resolution 2^-60 of max|f|, finer than FP64 for every |f| above 2^-7 of max|f|), and the
        F64 filter arithmetic without the IEEE decode/encode.  The API still takes and returns
        doubles.  Needs |f| < 2^Ef (else VLASOV_ERANGE).
   BF16: experiment: bfloat16 storage (8 significant bits, 2 bytes per cell), interpolation in FP32,
        displacements and moment sums as for F32.  Uploads round to nearest even.  Single grids
        only (not the batched form). */
enum { VLASOV_F64 = 0, VLASOV_F32 = 1, VLASOV_F64_NATIVE = 2, VLASOV_FX64 = 3, VLASOV_BF16 = 4 };

typedef struct vlasov_sim vlasov_sim; /* opaque; owns every device buffer it uses */

typedef struct {
    double xmin, xmax;   /* x (theta) domain; x_periodic=1 wraps it */
    double pmin, pmax;   /* momentum domain */
    int x_periodic;      /* 1: periodic; 0: f = 0 (and f'' = 0) outside the grid */
    int p_periodic;      /* same for p */
    double eps;          /* ring softening of Eq. (ringpot), > 0 for VLASOV_RING */
    double G;            /* sheet coupling: V(x) = 2 pi G |x| */
    int precision;       /* VLASOV_F64, VLASOV_F32, VLASOV_F64_NATIVE, VLASOV_FX64 or VLASOV_BF16 */
    void* stream;        /* cudaStream_t to enqueue on; NULL = a stream owned by the handle */
} vlasov_domain;

/* Moments of f after a full step (Sec. 4 diagnostics): mass = int f, Mx/My = int cos/sin(x) f
   (Eq. mxmydef), kinetic = int p^2/2 f, potential = 1/2 int int V(x-x') rho rho', energy = sum. */
typedef struct {
    double t, mass, Mx, My, kinetic, potential, energy;
    long long step;
} vlasov_moments_t;

/* Create a simulation on the current CUDA device.
   Nx, Np: multiples of 8, 16 <= N; Nx <= 8192 (x rows are staged whole in shared memory; 8-byte
   rows longer than 4096 cells take x-shift thread blocks of 512 threads, and the fused x-shifts
   then stay off).
   dt > 0.  domain: xmin < xmax, pmin < pmax; eps > 0 for the ring model.
   On success *out owns ~2*Nx*Np*sizeof(f) + O(Nx*#SM) bytes of device memory.
   Errors: VLASOV_EINVAL, VLASOV_ENOMEM, VLASOV_ECUDA. */
int vlasov_create(int model, int Nx, int Np, const vlasov_domain* domain, double dt,
                  vlasov_sim** out);

/* Upload f (host, Np*Nx doubles, f[j*Nx+i]); converts to the handle's precision (on the device
   for the 8-byte storage modes; page-locked host memory gives the full copy bandwidth).  Resets the
   step counter and the moment history.  Syncs. */
int vlasov_set_f(vlasov_sim* sim, const double* host_f);

/* Same from a device array of Np*Nx doubles (e.g. a torch tensor's data_ptr()).  Syncs (it reads
   back max|f| to set the scales of the fixed-point moment sums, as vlasov_set_f does).  The moment
   sums assume |f| stays below 4x the largest |f| uploaded. */
int vlasov_set_f_device(vlasov_sim* sim, const double* dev_f);

/* Write one of the waterbag initial states of Sec. 4 on the device (no host array), normalised to
   unit mass dx dp sum f = 1, on the nodes x_i = xmin + i dx, p_j = pmin + j dp:
     mode 0 (box, Secs. 4.1-4.3): f = 1/(4 x0 p0) where |x_i| < x0 and |p_j| < p0 (x0 >= half the x
       extent: every column, the homogeneous waterbag), times (1 + noise xi_ij), xi_ij = 2u - 1 with
       u the top 53 bits of the (j*Nx + i + 1)-th output of SplitMix64 started at `seed`;
     mode 1 (homogeneous waterbag with a cos mode, Sec. 4.2): f = [|p_j| < p0] / (2 p0 L)
       (1 + mode_amp cos x_i), L = xmax - xmin; `noise` and `seed` are not used.
   Arithmetic: the profile in FP64, each product rounded on its own (no fused multiply-add), the
   mass as an exact fixed-point sum rounded once, f = value / mass in FP64, then converted to the
   handle's storage as vlasov_set_f_device converts.  Same reset of step counter and history as
   vlasov_set_f.  Needs x0, p0 > 0, 0 <= noise < 1, |mode_amp| < 1 and a non-empty state on the
   grid (else VLASOV_EINVAL).  Allocates a temporary (Nx + Np) * 8 + 10 KB block while it runs.
   Syncs. */
int vlasov_init_waterbag(vlasov_sim* sim, double x0, double p0, double noise, unsigned long long seed, int mode,
                         double mode_amp);

/* Download the current f as doubles (host, Np*Nx).  Syncs.  VLASOV_ETIMEOUT if a device wait
   expired since the last check. */
int vlasov_get_f(vlasov_sim* sim, double* host_f);

/* Same into device memory (Np*Nx doubles).  Enqueued. */
int vlasov_get_f_device(vlasov_sim* sim, double* dev_f);

/* Enqueue n Strang steps (Sec. 3 steps 1-4).  Asynchronous: launches CUDA graphs on the handle's
   stream, one per run of 2^L steps (L < 6, largest runs first); the first call captures them for
   both ping-pong buffers (a few milliseconds of host time), later calls only launch.  The moments
   of f after each step are appended to a device ring of 4096 records.
   With fused x-shifts (vlasov_fused_x) a call of n >= 2 steps runs the second x half-shift of step
   k and the first of step k+1 as one launch that keeps the row between them on chip: the same
   arithmetic as separate launches, with one HBM round trip of f fewer per step.
   The state between calls is always a whole step. */
int vlasov_step(vlasov_sim* sim, int n);

/* Spline of every shift.  VLASOV_SPLINE_FD (default): the paper's method, f'' from the eighth-order
   9-point difference of Eq. (findif).  VLASOV_SPLINE_GS: the global cubic spline the paper compares
   it with (Sec. 3, Eq. tridiagsys; Tables 1-2): f'' solves the tridiagonal system of a line, cyclic
   on a periodic axis; on a zero-outside axis the natural spline through the data extended by zeros
   (f = f'' = 0 at the nodes next to the grid; the system's diagonal read as 2/3, the value the
   first-derivative continuity of its derivation gives).  GS runs in IEEE arithmetic of the storage
   type: VLASOV_F64_NATIVE or VLASOV_F32 storage, 64 <= Nx <= 8192, Np >= 64 (else VLASOV_EINVAL),
   and turns the fused x-shifts off.  Waits for the handle's stream; later steps and substeps use it.
   vlasov_spline reports the current choice. */
enum { VLASOV_SPLINE_FD = 0, VLASOV_SPLINE_GS = 1 };
int vlasov_set_spline(vlasov_sim* sim, int spline);
int vlasov_spline(const vlasov_sim* sim);

/* Turn the fused x-shifts on (1) or off (0).  Available with VLASOV_FX64 storage (Nx <= 4096 and
   a multiple of 64; on by default when x is periodic) and with VLASOV_F32 or VLASOV_BF16 storage
   (Nx <= 4096; on by default).  Elsewhere asking for them returns VLASOV_EINVAL.
   With FX64 the fused run gives the same bits as the separate launches; with FP32-class storage f
   is bitwise the same for a given force, but the per-CTA FP32 column and kinetic sums run over
   another row partition, so self-consistent runs agree to within the rounding of those sums.
   vlasov_fused_x reports the current setting (0 or 1). */
int vlasov_set_fused_x(vlasov_sim* sim, int on);
int vlasov_fused_x(const vlasov_sim* sim);

/* Method of the ring model's circulant convolutions, Eq. (ringpot) into Eq. (meanforce) (Sec. 2):
   F_i = -dx sum_k V'((i-k) dx) rho_k each step, and Phi_i = dx sum_k V((i-k) dx) rho_k for the
   potential energy U = 1/2 dx sum_i rho_i Phi_i of each moment record.
     VLASOV_RING_DIRECT:  N^2 fused multiply-adds in the storage's arithmetic type (FP64 for the
                          8-byte modes, FP32 for F32/BF16 storage).
     VLASOV_RING_FIXED:   the same sums exactly in integer arithmetic: rho as the exact fixed-point
                          column sums the x-shift produces, V' and V rounded to fixed point (relative
                          2^-52), int128 products and sums; FP64-accurate in every storage mode,
                          deterministic, and the same bits whatever the launch shape.  Default.
     VLASOV_RING_FFT:     FP64 FFT convolution in shared memory (Nx a power of two, <= 4096); the
                          potential by Parseval.  VLASOV_RING_FFT_F32: the same in FP32.
     VLASOV_RING_TENSOR:  the circulant product as a GEMM on the tensor cores (tcgen05, TF32 inputs
                          split in high and low parts, three products accumulated in FP32: about
                          FP32 accuracy); Nx = 128 k with 256 <= Nx <= 4096.
   vlasov_set_ring_method returns VLASOV_EINVAL for another model, an unknown method, or an Nx the
   method cannot take; it syncs and drops the captured step graphs.  vlasov_ring_method reports it
   (0 for another model).  vlasov_ring_timings computes the density of the current f and times
   `reps` force launches of each method that can run, with CUDA events on the handle's stream:
   us[m] = microseconds per launch of method m (us[0] and methods that cannot run: 0); us holds
   VLASOV_RING_METHODS doubles.  It leaves the method unchanged and overwrites only the force
   buffer.  Syncs. */
enum { VLASOV_RING_DIRECT = 1, VLASOV_RING_FIXED = 2, VLASOV_RING_FFT = 3, VLASOV_RING_FFT_F32 = 4,
       VLASOV_RING_TENSOR = 5, VLASOV_RING_METHODS = 6 };
int vlasov_set_ring_method(vlasov_sim* sim, int method);
int vlasov_ring_method(const vlasov_sim* sim);
int vlasov_ring_timings(vlasov_sim* sim, int reps, double* us);

/* Copy out up to max moment records produced since the previous call (oldest first) into out,
   set *count.  Records older than the ring's 4096 are dropped (count tells what is returned).
   Syncs; VLASOV_ETIMEOUT if a device wait expired. */
int vlasov_moments(vlasov_sim* sim, vlasov_moments_t* out, int max, int* count);

/* Test hooks (each syncs).
   vlasov_substep: one shift of the current f along axis 0 (x, rows) or 1 (p, columns) by the
     given displacements in cells (host; Np values for axis 0, Nx for axis 1): node i takes the
     spline value at i - disp.  Eqs. (step1)/(step3) with an arbitrary displacement.
   vlasov_density_force: density rho_i = dp sum_j f[j,i] and force F_i of Eq. (meanforce) for the
     current f (host outputs of Nx doubles; either may be NULL). */
int vlasov_substep(vlasov_sim* sim, int axis, const double* host_disp);
int vlasov_density_force(vlasov_sim* sim, double* host_rho, double* host_F);

/* Casimirs of the current f (Eq. casimirs, Sec. 4): *entropy = -dx dp sum over nodes with f > 0 of
   f ln f (s(f) = -f log f, the entropy whose loss measures the information lost to the grid;
   nodes where spline undershoot made f <= 0 add nothing) and *l2 = dx dp sum f^2 (s(f) = f^2);
   either pointer may be NULL.  FP64 arithmetic on the stored values, fixed summation order
   (deterministic).  Syncs. */
int vlasov_casimirs(vlasov_sim* sim, double* entropy, double* l2);

/* Check of the failure path (the paper has no failure handling; this exercises the library's own).
   Enqueues on the handle's stream one CTA that waits, with the bounded wait every staged sweep uses
   (a %globaltimer limit, 2 s in the sweeps), on an mbarrier that nothing arrives on and no copy
   completes, so the wait expires after limit_ns (1e3 <= limit_ns <= 2e9, else VLASOV_EINVAL); the
   CTA then records the timeout code in the handle's device error flag and returns.  Nothing is in
   flight while it waits, so the device context stays usable.  The next syncing call (vlasov_sync,
   vlasov_get_f, vlasov_moments, ...) returns VLASOV_ETIMEOUT and clears the flag; the state f is
   not touched.  Returns VLASOV_OK once enqueued. */
int vlasov_test_expire_wait(vlasov_sim* sim, long long limit_ns);

/* Wait for the handle's stream and report any device-side error flag. */
int vlasov_sync(vlasov_sim* sim);

/* Free every device resource of the handle (NULL is ignored). */
void vlasov_destroy(vlasov_sim* sim);

/* Message of the last failing call on this thread ("" if none). */
const char* vlasov_last_error(void);

/* Kernel launches per step in a long run (the slots of vlasov_step_timed), and the exact number
   that vlasov_step(n) enqueues (for launch accounting). */
int vlasov_kernels_per_step(const vlasov_sim* sim);
long long vlasov_launches(const vlasov_sim* sim, int n);

/* Run n steps with eager launches (no graph) and a CUDA event around every kernel, on the handle's
   stream; ms_per_launch[q] receives the mean duration of launch slot q of a step (q <
   vlasov_kernels_per_step; max_launches must be at least that), *nlaunch the slot count.  Syncs.
   Without fused x-shifts (or n = 1) the slots of each of the n steps, in order: x-shift (step 1,
   density partials), density reduction, [ring force], p-shift filters (force), p-shift (step 3),
   x-shift (step 4, density+kinetic partials), moment reduction, [ring potential].  HMF with
   VLASOV_FX64, VLASOV_F32 or VLASOV_BF16 storage (Nx * Np <= 2^24, spline of Eq. findif) has no
   density reduction launch: the x-shifts hand the reductions three exact per-CTA numbers and the
   filters launch forms Mx, My.
   With fused x-shifts and n >= 2 the slots are those between two steps, averaged over the n-1 such
   places: fused x-shifts (step 4 and the next step 1), moment reduction, [ring potential],
   [density reduction, ring force], p-shift filters, p-shift.  The ring with VLASOV_RING_FIXED
   merges the two reductions into one launch and the two convolutions (the end state's potential,
   the next force) into another: fused x-shifts, reductions, convolutions, filters, p-shift. */
int vlasov_step_timed(vlasov_sim* sim, int n, double* ms_per_launch, int max_launches, int* nlaunch);

/* ---------------------------------------------------------------------------------------------
   Batched form and serving.  Many simulations of different models, grid sizes, initial states and
   step counts advance together: each kernel of a Strang step is launched once for all of them
   (FP32 or FX64 storage of f, FP64-accurate displacements and moment sums), from one captured
   CUDA graph.
   p is always f = 0 outside in the batched form.  Results of a simulation do not depend on which
   others share the batch (each keeps its own fixed CTA-to-row mapping; sums are order-free). */
typedef struct vlasov_batch vlasov_batch;

typedef struct {
    int model;                   /* VLASOV_HMF, VLASOV_RING, VLASOV_SHEET, VLASOV_FREE */
    int Nx, Np;                  /* multiples of 8, 16 <= N <= the batch's max_n */
    double xmin, xmax, pmin, pmax;
    int x_periodic;              /* 0: f = 0 outside in x (|x displacement| must stay <= 55 cells) */
    double eps, G, dt;           /* ring softening, sheet coupling, time step */
    int init;                    /* 0: f = c [|x|<x0][|p|<p0] (1 + noise xi), xi = 2u-1 from SplitMix64
                                       output j*Nx+i+1 of `seed` (x0 >= half the x extent: all columns);
                                    1: f = c [|p|<p0] (1 + amp cos x); both renormalised to unit mass */
    double x0, p0, noise, amp;
    unsigned long long seed;
    int steps;                   /* Strang steps to run */
    double arrival_s;            /* vlasov_serve: arrival time after the start of the run */
} vlasov_request;

typedef struct {
    int status;                  /* 0 done; VLASOV_E* if it could not run (1: still pending) */
    int steps;
    double arrival_s, admit_s, done_s;   /* done_s: when the GPU finished its last step */
    vlasov_moments_t last;       /* moments after the last step */
    vlasov_moments_t first;      /* moments after the first step */
} vlasov_result;

/* A batch of `slots` simulation slots with grids up to max_n x max_n, all buffers carved out of one
   device allocation of mem_budget_bytes (admission fails with VLASOV_ENOMEM while a request does not
   fit).  precision: VLASOV_F32 (FP32 storage) or VLASOV_FX64 (the FP64-accurate 64-bit fixed-point
   storage of the single-grid VLASOV_FX64 mode, same kernels: a slot's f is bit-identical to a
   single-grid VLASOV_FX64 run of the same request and f0), for every slot; max_n <= 4096 for FX64.
   stream: cudaStream_t or NULL for an owned one.  VLASOV_EINVAL for other precisions. */
int vlasov_batch_create(int slots, int max_n, long long mem_budget_bytes, int precision, void* stream,
                        vlasov_batch** out);

/* Launch shape of the batched sweeps.  rows_per_cta: x-shift rows per CTA (a slot with Np rows runs
   on clamp(ceil(Np / rows_per_cta), 16, 512) CTAs, whatever else is in the batch); tiles_per_cta:
   p-shift tiles (32 columns x 128 rows; 112 rows with VLASOV_FX64) per CTA of the batch's largest grid (each slot's p-shift
   launch has clamp(tiles / tiles_per_cta, 32, 1024) CTAs). */
typedef struct {
    int rows_per_cta;
    int tiles_per_cta;
} vlasov_batch_shape;

/* As vlasov_batch_create with an explicit shape (NULL: the tuned shape for (max_n, precision) if
   vlasov_batch_autotune ran for it in this process, else {16, 8}).  rows_per_cta in 1..4096,
   tiles_per_cta in 1..1024, else VLASOV_EINVAL.  With VLASOV_FX64 a slot's results do not depend
   on the shape (exact fixed-point sums); with VLASOV_F32 they move at rounding level (each CTA's
   FP64 column and kinetic sums are rounded before the exact sum over CTAs).  Within one batch the
   shape is fixed, so a slot's results never depend on the rest of the batch. */
int vlasov_batch_create_shaped(int slots, int max_n, long long mem_budget_bytes, int precision, void* stream,
                               const vlasov_batch_shape* shape, vlasov_batch** out);
int vlasov_batch_shape_of(const vlasov_batch* b, vlasov_batch_shape* out);

/* Autotuner of the batched launch shape: times every candidate (rows_per_cta in {8, 16, 32, 64} x
   tiles_per_cta in {2, 4, 8, 16}, in that order, tiles fastest) on this GPU with a batch of eight
   synthetic HMF requests (two each of max_n, max_n/2, max_n/4, max_n/8, at least 16) for 8 batched
   steps after 2 warm-up steps, returns the fastest in *best and, if ms_per_step is not NULL, the
   16 candidates' milliseconds per batched step (0 for a candidate that could not run).  The
   result is kept for the process: later batches of this (max_n, precision) use it.  Needs about
   2.5 x the device memory of those eight requests; syncs; a few seconds. */
int vlasov_batch_autotune(int max_n, int precision, void* stream, vlasov_batch_shape* best, double* ms_per_step);
/* Device bytes one request occupies in a batch of the given precision. */
long long vlasov_batch_footprint(const vlasov_request* req, int precision);
/* Admit a request into a free slot (*slot); host_f0 (Np*Nx doubles) or NULL for the device-side
   initial state of req->init.  VLASOV_ESTATE: no free slot; VLASOV_ENOMEM: does not fit now. */
int vlasov_batch_admit(vlasov_batch* b, const vlasov_request* req, const double* host_f0, int* slot);
/* Launch n batched steps; each slot stops at its own step count.  Asynchronous. */
int vlasov_batch_step(vlasov_batch* b, int n);
int vlasov_batch_slot_steps(vlasov_batch* b, int slot, int* steps_done);
/* Syncs; f as doubles (host, may be NULL) and up to max per-step moment records (oldest first). */
int vlasov_batch_get(vlasov_batch* b, int slot, double* host_f, vlasov_moments_t* moments, int max, int* count);
/* Free a slot and its memory (waits for work in flight). */
int vlasov_batch_release(vlasov_batch* b, int slot);
void vlasov_batch_destroy(vlasov_batch* b);

typedef struct {
    int slots;                   /* concurrent simulations */
    int max_n;                   /* largest grid (0: from the requests) */
    long long mem_budget_bytes;  /* device memory for simulation state */
    int max_inflight;            /* batched steps queued ahead of the GPU */
    int precision;               /* VLASOV_F32 or VLASOV_FX64 */
    void* stream;
    int autotune;                /* 1: vlasov_batch_autotune for (max_n, precision) before the run */
} vlasov_serve_options;

/* Continuous-batching run of a request stream: requests are admitted (in arrival order, at their
   arrival time on the wall clock) as slots and memory free up, advance together one batched step at
   a time, and retire independently.  results[i] belongs to reqs[i].  *makespan_s: wall time.
   precision other than VLASOV_F32 or VLASOV_FX64: VLASOV_EINVAL. */
int vlasov_serve(const vlasov_request* reqs, int n, const vlasov_serve_options* opt, vlasov_result* results,
                 double* makespan_s);

/* One x-shift sweep (node i of row j takes the spline value at i - dev_disp[j]) with its density,
   for callers that cannot allocate device memory.  The paper has no counterpart: this exists because
   some callers may not call cudaMalloc at all (a host callback or allocator hook, a framework that
   owns every device allocation, a plug-in that must keep its device footprint fixed after load).
   It allocates nothing: its scratch (row filters and column partial sums, about 5.1 MiB) is a
   fixed array inside the library that every GPU loading the library holds until process exit.
   dev_fin, dev_fout: Np*Nx doubles (f[j*Nx+i], device, caller-owned, must not overlap);
   dev_rho: Nx doubles out, rho_i = dp * sum_j fout[j,i] with dp = (pmax-pmin)/Np;
   dev_disp: Np doubles (device).  Limits: 16 <= Nx, Np <= 4096, multiples of 8; with
   x_periodic = 0 every displacement s must satisfy -57 < s <= 56 (the foot cell floor(-s) at most
   56 cells away; the fixed zero halo is 64 cells).  A displacement out of range (or NaN), or a
   bounded device wait that gives up, makes dev_rho all NaN.  FP64 only.
   Enqueued on `stream` (NULL = legacy default stream); returns VLASOV_EINVAL/ECUDA on bad input.
   The first call on a device looks up the scratch address and sets kernel attributes for that
   device; make that first call outside any stream capture.  Every call shares the one scratch
   array: calls that overlap on the GPU (other streams, other threads) race and must not be
   issued; keep them ordered on one stream. */
int vlasov_xshift_density_noalloc(const double* dev_fin, double* dev_fout, double* dev_rho, int Nx, int Np,
                                  double pmin, double pmax, int x_periodic, const double* dev_disp,
                                  void* stream);

#ifdef __cplusplus
}
#endif
#endif
