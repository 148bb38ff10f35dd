/*
 * tacaw.h -- C ABI of libtacaw.so, the GB300 (sm_103a) TACAW hot path.
 *
 * The method is the one of arXiv 2602.10064 (PySlice): for every frame of an atomic
 * trajectory and every probe position the electron wave is propagated by multislice
 * through slice potentials built from Kirkland's parametrisation, and the stack of exit
 * waves psi(k, t) is transformed along time to give the vibrational intensity
 * I(k, w) = |F_t[psi(k,t) - <psi(k,t)>_t]|^2.
 *
 * Conventions shared by every call:
 *  - Every call returns an int: TACAW_OK (0) or a negative TACAW_E* code.  The message of the
 *    last failure on a context is available from tacaw_last_error().  A failed call leaves
 *    output buffers unspecified and the context usable.
 *  - Device pointers are plain CUDA device addresses (e.g. torch tensor data_ptr()).  The
 *    caller owns every buffer it passes; the library owns the context, its tables, its
 *    scratch memory and the state of admitted serving requests.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls taking a
 *    stream are stream-ordered and asynchronous unless stated otherwise: they return once the
 *    work is enqueued.  Scratch memory comes from the stream-ordered allocator of the context's
 *    device and is released on the same stream.
 *  - Arrays are row-major, complex values are interleaved (re, im) float32 pairs ("c64").
 *    Reciprocal-space arrays are in FFT order: index i on an n-point axis of length L has
 *    spatial frequency k = m / L (cycles per Angstrom, no 2 pi) with m = i for i < (n+1)/2
 *    and m = i - n otherwise.  Time-frequency bins are in the same order: bin m has
 *    f_m = m / (F dt).
 *  - Grids nx, ny must be powers of two in [32, 1024], or one of 96, 192, 384, 768 (3 * 2^k)
 *    and 1152 (9 * 2^7: 0.1 A sampling of a ~110 A cell).
 *  - Units: Angstrom, eV, fs, mrad; potentials in V*A (projected), sigma in rad/(V*A).
 */
#ifndef TACAW_H
#define TACAW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TACAW_OK 0
#define TACAW_PENDING 1      /* tacaw_poll: request admitted or queued, not finished */
#define TACAW_EINVAL (-1)    /* bad argument: shape, size, pointer kind, unknown species */
#define TACAW_ENOMEM (-2)    /* device allocation failed */
#define TACAW_ETOOBIG (-3)   /* request can never fit the context's HBM budget */
#define TACAW_ETIMEOUT (-4)  /* a bounded wait ran out (kernel status word or tacaw_wait) */
#define TACAW_ECUDA (-5)     /* CUDA runtime error; see tacaw_last_error */
#define TACAW_ECANCELED (-6) /* request cancelled before it finished */
#define TACAW_ENOTFOUND (-7) /* unknown ticket */

/* Time-transform arithmetic (tacaw_spectrum, tacaw_run). */
#define TACAW_DFT_FP32 0   /* FP32 SIMT dense DFT: the plain path */
#define TACAW_DFT_BF16X3 1 /* tcgen05 BF16 GEMM, hi*hi + hi*lo + lo*hi, FP32 accumulation */
#define TACAW_DFT_TF32X3 2 /* tcgen05 TF32 GEMM, same three-product split */
#define TACAW_DFT_BF16 3   /* tcgen05 BF16 GEMM, single product (precision study only) */
#define TACAW_DFT_TF32 4   /* tcgen05 TF32 GEMM, single product (precision study only) */

/* Output reduction (tacaw_spectrum, tacaw_run). */
#define TACAW_REDUCE_NONE 0     /* full S[P][F][ny][nx] */
#define TACAW_REDUCE_DETECTOR 1 /* spectrum image SI[P][F] = sum over the band-limited disc of S */

typedef struct tacaw_ctx tacaw_ctx;

/* Geometry and beam of one simulation. */
typedef struct tacaw_params {
  int32_t nx, ny;                 /* grid points along x and y */
  int32_t n_slices;               /* S >= 1; slice thickness dz = cell[2] / S */
  int32_t bandlimit_transmission; /* 1: t <- IDFT(M DFT(t)) / Nq; 0: t = exp(i sigma V) */
  double cell[3];                 /* periodic cell Lx, Ly, Lz (A) */
  double voltage_ev;              /* beam energy (eV) */
  double bandlimit;               /* mask radius as a fraction of Nyquist (2/3); <= 0: no mask */
  double dt_fs;                   /* frame spacing (fs); sets the frequency axis only */
} tacaw_params;

/* Illumination (Discussion, "Beyond Vibrational Spectroscopy": aberration function applied
 * at probe formation, with defocus, astigmatism, coma and spherical aberration; arbitrary
 * complex wavefronts).  A convergent probe is
 * psi0(k) = A(k) exp(-i chi(k)) exp(-2 pi i k.r_p) / norm with A = 1 for |k| <= alpha/lambda and
 * chi(k) = pi lambda k^2 (defocus + astig cos 2(phi_k - astig_angle))
 *        + (2 pi / 3) coma lambda^2 k^3 cos(phi_k - coma_angle) + (pi/2) Cs lambda^3 k^4,
 * i.e. (2 pi / lambda) (C1 theta^2 / 2 + C21 theta^3 / 3 + C3 theta^4 / 4) at theta = lambda k, so
 * a positive defocus equals free propagation over that distance. */
typedef struct tacaw_probe {
  double alpha_mrad;   /* convergence semi-angle; <= 0: plane wave (n_probes must be 1) */
  int32_t n_probes;    /* P >= 1 */
  int32_t pad_;
  const double* xy;    /* HOST [P][2] probe positions (A); NULL: all probes at (0, 0) */
  double defocus;      /* A */
  double cs_mm;        /* spherical aberration, mm */
  double astig;        /* two-fold astigmatism, A */
  double astig_angle;  /* rad */
  const float* psi0;   /* DEVICE c64 [P][ny][nx]: real-space initial waves to use instead of the
                          aperture probe (e.g. vortex beams), normalised by the caller; NULL: none */
  double coma;         /* axial coma C21, A */
  double coma_angle;   /* rad */
} tacaw_probe;

/* Library version string (static storage). */
const char* tacaw_version(void);

/* Sampling of a simulation (Supplement, "Sampling Considerations": reciprocal-space resolution
 * dk = 1/L, reach k_max = 1/(2 dx); frequency resolution df = 1/(F dt), Nyquist f_max =
 * 1/(2 dt)).  Host-only arithmetic, no context and no GPU.  Outputs (HOST, any may be NULL):
 * kx [nx] and ky [ny], the spatial frequencies (1/A) of the grid in FFT order; f_thz [n_frames],
 * the frequencies of the time-transform bins in FFT order (THz); sampling [6] = dk_x, dk_y,
 * k_max_x, k_max_y (1/A), df, f_max (THz).  Uses nx, ny, cell[0..1] and dt_fs of params.
 * EINVAL for sizes below 1 or non-positive lengths or dt. */
int tacaw_axes(const tacaw_params* params, int64_t n_frames, double* kx, double* ky, double* f_thz,
               double* sampling);

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the device memory the
 * serving loop admits at once (0 = 90% of the device's free memory at creation).  *out
 * receives a library-owned handle, released by tacaw_destroy. */
int tacaw_create(tacaw_ctx** out, int32_t device, uint64_t hbm_budget_bytes);

/* Destroy a context: waits for admitted serving requests, frees every library allocation. */
int tacaw_destroy(tacaw_ctx* ctx);

/* Message of the last failure on ctx (empty string if none); valid until the next call. */
const char* tacaw_last_error(const tacaw_ctx* ctx);

/* Load form-factor coefficients (Methods, "Atomic Scattering Potentials": Kirkland's form
 * f(q) = sum_i a_i/(q^2+b_i) + c_i exp(-d_i q^2), q in 1/A without 2 pi, f in A).
 * Z: HOST [nZ] atomic numbers; coef: HOST [nZ][12] as a1 b1 a2 b2 a3 b3 c1 d1 c2 d2 c3 d3.
 * Replaces any earlier table.  EINVAL for nZ < 1, nZ > 64, Z outside [1, 255], repeated Z
 * or b_i <= 0. */
int tacaw_load_form_factors(tacaw_ctx* ctx, const int32_t* Z, const double* coef, int32_t nZ);

/* Slice binning (Methods, "Atomic Scattering Potentials": the sum runs over the atoms inside
 * a slice's z-bounds).  slice_out[f][j] = s with z wrapped into [0, Lz) and
 * s = floor(z_w / dz) clamped to [0, S-1], all in FP64 from the float32 input.
 * pos: DEVICE float32 [nf][n_atoms][3]; slice_out: DEVICE int32 [nf][n_atoms]. */
int tacaw_bin_slices(tacaw_ctx* ctx, const tacaw_params* params, const float* pos, int64_t n_atoms,
                     int64_t nf, int32_t* slice_out, void* stream);

/* Projected potential of every slice of nf frames (Methods, "Atomic Scattering Potentials"):
 * V_s(r) = sum_k (2 pi a0 e / A) M(k) sum_{j in s} f_Zj(|k|) exp(2 pi i k.(r - r_j)), A = Lx Ly.
 * The structure factor is evaluated by spreading each atom onto the grid with an
 * exponential-of-semicircle kernel (width 12, beta 24) and deconvolving after the FFT.
 * pos: DEVICE float32 [nf][n_atoms][3] (A); Z: DEVICE int32 [n_atoms] (each Z must be in the
 * loaded table); V_out: DEVICE float32 [nf][S][ny][nx] (V*A).  The spread structure factor is
 * accurate only inside a band limit of at most 2/3 of Nyquist; EINVAL for bandlimit <= 0 or
 * > 2/3 (the same holds for tacaw_run). */
int tacaw_build_potential(tacaw_ctx* ctx, const tacaw_params* params, const float* pos, const int32_t* Z,
                          int64_t n_atoms, int64_t nf, float* V_out, void* stream);

/* Transmission functions (Methods, "Multislice Propagation": t = exp(i sigma V)), optionally
 * band-limited.  V: DEVICE float32 [nf][S][ny][nx]; t_out: DEVICE c64 [nf][S][ny][nx]. */
int tacaw_transmission(tacaw_ctx* ctx, const tacaw_params* params, const float* V, int64_t nf,
                       float* t_out, void* stream);

/* Multislice (Methods, "Multislice Propagation"): for each probe p and frame f,
 * psi <- IDFT(P M DFT(t_s psi)) / Nq for s = 0..S-1 with P(k) = exp(-i pi lambda dz |k|^2),
 * then psi_k = DFT(psi_exit) / sqrt(Nq).  V: DEVICE float32 [nf][S][ny][nx];
 * psi_k_out: DEVICE c64 [P][nf][ny][nx]. */
int tacaw_propagate(tacaw_ctx* ctx, const tacaw_params* params, const float* V, int64_t nf,
                    const tacaw_probe* probe, float* psi_k_out, void* stream);

/* Time transform (Methods, "Workflow Architecture"): for every (p, q)
 * S[p][m][q] = |sum_n (psi[p][n][q] - mean_n psi[p][n][q]) exp(-2 pi i m n / F)|^2,
 * the mean and the residual to FP64-class precision (FP32-pair sums and exact differences,
 * combined in FP64 once per q), the sum by the arithmetic `precision` (TACAW_DFT_*).
 * psi_k: DEVICE c64 [P][F][nq]; q_sel: DEVICE int32 [n_sel] ascending q indices to transform
 * (others are written as 0), or NULL for all nq; S_out: DEVICE float32 [P][F][nq] for
 * TACAW_REDUCE_NONE or [P][F] (sum over the selected q) for TACAW_REDUCE_DETECTOR. */
int tacaw_spectrum(tacaw_ctx* ctx, const float* psi_k, int64_t P, int64_t F, int64_t nq, int32_t precision,
                   int32_t reduce, const int32_t* q_sel, int64_t n_sel, float* S_out, void* stream);

/* The whole hot path for one trajectory, fused: binning, potential, transmission,
 * multislice for every (probe, frame), time transform over the band-limited q only.
 * pos: float32 [F][n_atoms][3] and Z: int32 [n_atoms], HOST or DEVICE; S_out: float32
 * [P][F][ny][nx] (REDUCE_NONE) or [P][F] (REDUCE_DETECTOR), HOST or DEVICE.  With host
 * buffers the copies are part of the call (pinned host memory is fastest).  Synchronous on
 * `stream` when any buffer is on the host, asynchronous otherwise.  Z on the device is mapped
 * to form-factor slots on the device: an atom whose Z is not in the loaded table makes the
 * next tacaw_check return TACAW_EINVAL (the results of that call are invalid); Z on the host
 * is checked here (TACAW_EINVAL). */
int tacaw_run(tacaw_ctx* ctx, const tacaw_params* params, const float* pos, const int32_t* Z, int64_t n_atoms,
              int64_t n_frames, const tacaw_probe* probe, int32_t precision, int32_t reduce, float* S_out,
              void* stream);

/* ---- TACAW accessors and trajectory averaging ------------------------------------------------ */

/* Spectral diffraction (Methods, "Data Structure Design": I(k, w) at one frequency):
 * out[p][q] = S[p][m][q] with m = round(f_thz F dt_fs 1e-3) mod F (FFT order), plus S[p][-m][q]
 * when fold != 0 (energy loss and gain together).  S: DEVICE float32 [P][F][nq]; out: DEVICE
 * float32 [P][nq].  With the detector-summed SI[P][F] of tacaw_spectrum (nq = 1) this is the
 * spectrum image at f. */
int tacaw_spectral_diffraction(tacaw_ctx* ctx, const float* S, int64_t P, int64_t F, int64_t nq, double dt_fs,
                               double f_thz, int32_t fold, float* out, void* stream);

/* Dispersion along a reciprocal-space path (same section, "dispersion()"): S[p][m] bilinearly
 * interpolated at the points (kx, ky) (1/A, HOST [npts] each) on the periodic k grid of spacing
 * (1/Lx, 1/Ly).  S: DEVICE float32 [P][F][ny][nx]; out: DEVICE float32 [P][F][npts]. */
int tacaw_dispersion(tacaw_ctx* ctx, const float* S, int64_t P, int64_t F, int32_t ny, int32_t nx, double Lx,
                     double Ly, const double* kx, const double* ky, int32_t npts, float* out, void* stream);

/* Trajectory averaging (Supplement, "Sampling Considerations": average the spectra of
 * independent trajectories): acc[i] += weight * S[i] in FP64.  S: DEVICE float32 [n];
 * acc: DEVICE float64 [n]. */
int tacaw_accumulate(tacaw_ctx* ctx, const float* S, int64_t n, double weight, double* acc, void* stream);

/* ---- one trajectory split by frames across processes --------------------------------------- */

/* In-band q points of a geometry: the q = y nx + x inside the 2/3-disc band limit (all q
 * without one), ascending, that tacaw_run transforms.  *n_out receives their count; q_out
 * (HOST int32, may be NULL) receives the list. */
int tacaw_band_points(tacaw_ctx* ctx, const tacaw_params* params, int32_t* q_out, int64_t* n_out);

/* Partial time transform of the frames [f0, f0 + nf) of an F-frame trajectory (Supplement,
 * "Sampling Considerations": frames are independent until the time transform), for a
 * trajectory split by frames across processes:
 *   psi_tilde[p][m][j] = sum_{n < nf} exp(-2 pi i m (f0 + n) / F) (psi[p][n][q_j] - psi_ref[p][q_j]).
 * Subtracting a time-independent reference instead of the frame mean (Methods, "Workflow
 * Architecture") changes the transform only at m = 0, so the sum of the partial transforms of
 * all processes (one all-reduce) gives every m != 0 bin; every process can use the exit wave
 * of the trajectory's first frame as psi_ref without communication.  FP32 arithmetic.
 * psi_k: DEVICE c64 [P][nf][nq]; psi_ref: DEVICE c64 [P][nq]; q_sel: DEVICE int32 [n_sel]
 * (NULL: all nq); psi_tilde: DEVICE c64 [P][F][n_sel], overwritten.  EINVAL for f0 < 0,
 * f0 + nf > F, sizes below 1, P or nf above 65535. */
int tacaw_spectrum_partial(tacaw_ctx* ctx, const float* psi_k, int64_t P, int64_t nf, int64_t f0, int64_t F,
                           int64_t nq, const float* psi_ref, const int32_t* q_sel, int64_t n_sel, float* psi_tilde,
                           void* stream);

/* Intensity of a summed transform: S[p][m][q_j] = |psi_tilde[p][m][j]|^2 with S = 0 at m = 0
 * (the mean-subtracted transform vanishes there), other q of S zero (TACAW_REDUCE_NONE;
 * S_out DEVICE float32 [P][F][nq], nq = n_sel without q_sel), or the spectrum image
 * SI[p][m] = sum_j S (TACAW_REDUCE_DETECTOR; S_out [P][F], FP64 sums). */
int tacaw_intensity(tacaw_ctx* ctx, const float* psi_tilde, int64_t P, int64_t F, int64_t n_sel,
                    const int32_t* q_sel, int64_t nq, int32_t reduce, float* S_out, void* stream);

/* ---- serving: requests admitted by device-memory footprint, run concurrently ------------ */

/* One TACAW simulation request: the inputs and output of tacaw_run. */
typedef struct tacaw_request {
  tacaw_params params;
  tacaw_probe probe;     /* n_probes = 0 means one plane wave; xy (host) is copied at submission */
  const float* pos;      /* HOST or DEVICE float32 [F][A][3]: host data is copied at submission,
                            device data must stay valid until the request has finished */
  const int32_t* Z;      /* HOST or DEVICE int32 [A], copied at submission */
  int64_t n_atoms;
  int64_t n_frames;
  int32_t precision;     /* TACAW_DFT_* */
  int32_t reduce;        /* TACAW_REDUCE_* */
  float* S_out;          /* HOST or DEVICE output laid out as in tacaw_run; written before the
                            request reports TACAW_OK and must stay valid until then */
} tacaw_request;

/* State of a request.  Times are seconds on the library's monotonic clock. */
typedef struct tacaw_result {
  int32_t status;             /* TACAW_PENDING while queued or running, then TACAW_OK or an error */
  int32_t batched;            /* requests in the run this one was part of (1: alone; see tacaw_submit) */
  uint64_t footprint_bytes;   /* device memory reserved for the request while it runs */
  double t_submit, t_admit, t_done;
} tacaw_result;

/* Queue a request (non-blocking).  The request is checked now (EINVAL as tacaw_run; ETOOBIG if
 * its footprint exceeds the context's budget).  A worker thread admits queued requests while
 * their footprints fit the budget and one of the context's serving streams (option
 * "serving_streams") is free, and runs
 * each on its own stream, so admitted requests overlap on the GPU; later requests are admitted
 * as memory frees up.  A request that does not fit can be overtaken by smaller ones at most 8
 * times.  Queued requests of the same geometry (parameters, probes, frame and atom counts,
 * species, arithmetic and output; positions may differ) are coalesced, up to 16 (option
 * "max_coalesce"), into one run
 * whose launches cover all of them; each result is the same, bit for bit, as alone.  *ticket
 * identifies the request. */
int tacaw_submit(tacaw_ctx* ctx, const tacaw_request* req, uint64_t* ticket);

/* Device bytes the request would reserve while it runs (its admission footprint), without
 * submitting it: *bytes is set and TACAW_OK returned if the request fits the context's budget,
 * TACAW_ETOOBIG if it never can; EINVAL as tacaw_submit (the buffer pointers are not needed).
 * A run bounds its scratch: probes are propagated and transformed in blocks, and a probe's
 * exit-wave stack keeps only the in-band points, so a scan's footprint grows with the block,
 * not with the number of probes. */
int tacaw_request_footprint(tacaw_ctx* ctx, const tacaw_request* req, uint64_t* bytes);

/* TACAW_PENDING while the request is queued or running; otherwise its final status (TACAW_OK,
 * an error code, or TACAW_ECANCELED), after which the ticket is released.  out (optional)
 * receives the request's state.  TACAW_ENOTFOUND for unknown or released tickets. */
int tacaw_poll(tacaw_ctx* ctx, uint64_t ticket, tacaw_result* out);

/* Block until the request finishes or timeout_s passes (< 0: no limit); returns as
 * tacaw_poll, or TACAW_ETIMEOUT (ticket kept) when the time ran out. */
int tacaw_wait(tacaw_ctx* ctx, uint64_t ticket, double timeout_s, tacaw_result* out);

/* Cancel a request: a queued one finishes at once with TACAW_ECANCELED; a running one runs to
 * the end but reports TACAW_ECANCELED (its host output is not written). */
int tacaw_cancel(tacaw_ctx* ctx, uint64_t ticket);

/* Hold (hold != 0) or release (0) admission: while held, submitted requests queue and none is
 * admitted (running ones continue).  Releasing admits the queue at once, and queued requests of
 * one geometry are coalesced into shared runs (up to the option "max_coalesce"), so a caller
 * that submits a batch between hold and release gets the batch's runs stacked.  Requests still
 * queued when the context is destroyed finish with TACAW_ECANCELED.  TACAW_EINVAL for a null
 * context. */
int tacaw_serving_hold(tacaw_ctx* ctx, int32_t hold);

/* Current serving load: queued and running requests, reserved and budgeted device bytes. */
int tacaw_serving_stats(tacaw_ctx* ctx, int64_t* queued, int64_t* active, uint64_t* used_bytes,
                        uint64_t* budget_bytes);

/* Allocation-free time transform.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- for example a host application that reserves
 * the device's memory for its own allocator up front, or that hands this library only the input
 * and output buffers under a fixed memory budget -- so neither a context (whose creation
 * allocates) nor cudaMalloc / cudaFree / an allocating library routine is used.
 * It computes the same S as tacaw_spectrum(..., TACAW_DFT_FP32, TACAW_REDUCE_NONE, q_sel = NULL):
 * S[p][m][q] = |sum_n (psi[p][n][q] - mean_n psi[p][n][q]) exp(-2 pi i m n / F)|^2 with the mean
 * and the residual to FP64-class precision (FP32-pair sums and exact differences, combined in
 * FP64 once per q) and the sum in FP32.
 * psi_k: DEVICE c64 [P][F][nq]; S_out: DEVICE float32 [P][F][nq], both on the current device;
 * stream as elsewhere.
 * Scratch (time twiddles, FP64 mean, residual: 8 F + 16 P nq + 8 P F nq bytes, each part
 * rounded up to 256 bytes) lives in a file-scope device array of 16 MiB that every GPU loading
 * the library holds until the process exits.  Larger problems return TACAW_ETOOBIG; P or F
 * above 65535, a NULL pointer, a pointer that is not device memory of the current device, or a
 * size below 1 return TACAW_EINVAL; a failed launch returns TACAW_ECUDA.  Every call looks up
 * the array's device address in the current context (cudaGetSymbolAddress, which allocates
 * nothing); the first lookup in a context can load the library's device code, so make the
 * first call on a device before any stream capture.  Every call overwrites all the scratch it
 * reads, so nothing carries over between calls, but all calls share the one array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be serialised by the
 * caller. */
int tacaw_spectrum_static(const float* psi_k, int64_t P, int64_t F, int64_t nq, float* S_out, void* stream);

/* Context option.  "max_chunk_frames": cap on the frames whose waves are propagated together
 * in one batch of launches (0 = automatic: a bounded scratch of 2 GB per chunk; 1 gives the
 * plain frame-at-a-time path).  "max_slice_block": cap on the slices whose potentials and
 * transmission functions tacaw_run builds together for a chunk of frames (0 = automatic: all
 * S slices unless that would leave a slice launch with fewer than "min_wave_rows" wave rows,
 * default 65536).  "max_run_bytes": bound on the scratch of one run (0 = automatic: half the
 * context's budget, at most 64 GiB); probes are propagated and transformed in blocks sized to
 * it.  "max_probe_block": cap on the probes of one block (0 = no cap).  "max_coalesce": the most
 * queued serving requests of one geometry coalesced into one run (default 16; 1 = none).
 * "serving_streams": streams per request class on which admitted serving requests run
 * concurrently (default 4; before the first tacaw_submit only).  "serving_small_work": requests
 * whose work (probes x frames x slices x nx x ny) is at most this (default 2^33) run on
 * high-priority streams of their own, so they wait neither for long requests' streams nor for
 * their pending blocks; the others on normal-priority streams.  "host_copy": how results reach
 * page-locked host memory (tacaw_run's S_out, serving requests' host outputs): 1 (default) by
 * SM stores into the mapped pages, 0 by the copy engine (cudaMemcpyAsync); pageable host
 * memory always goes through the copy engine.  "static_band": 1 (default) runs the row passes that
 * read or write in-band rows (spreading, potential output, the later slices) with kernels built
 * for the standard 2/3 band of a square cell when the run's band is that one; 0 always reads
 * the band at run time.
 * Results do not depend on these options.  EINVAL for an unknown name or a bad value. */
int tacaw_set_option(tacaw_ctx* ctx, const char* name, int64_t value);

/* Wait for all work on the context's device, then report what the context's kernels flagged
 * since the last check: TACAW_ETIMEOUT if a kernel gave up a bounded wait, TACAW_EINVAL if
 * tacaw_run met a device-resident Z that is not in the form-factor table (the outputs of
 * those calls are invalid), else TACAW_OK.  The status is cleared by the check. */
int tacaw_check(tacaw_ctx* ctx);

/* Self-test of the failure path of the bounded waits (the paper has no counterpart): one
 * kernel thread waits on a shared-memory barrier that nothing completes, gives up after
 * timeout_ms (0 < timeout_ms <= 1000) through the same bounded-wait routine the tensor-core
 * time transform uses, sets the status word and returns; the next tacaw_check then reports
 * TACAW_ETIMEOUT and the context stays usable.  No copy or MMA is in flight during the wait. */
int tacaw_selftest_wait(tacaw_ctx* ctx, double timeout_ms, void* stream);

/* Diagnostics.  tacaw_profile_begin starts recording a CUDA event pair around every kernel
 * launch of the calls that follow, on the stream each launch uses.  tacaw_profile_end stops,
 * waits for the recorded events and reports per kernel class i < max_n (in first-launch order):
 * its name (NUL-terminated, at most 31 characters, at names + 32 i), total milliseconds,
 * launch count, and the algorithmic bytes and flops those launches account for.  *n_out
 * receives the number of classes.  Any output pointer may be NULL. */
int tacaw_profile_begin(tacaw_ctx* ctx);
int tacaw_profile_end(tacaw_ctx* ctx, char* names, double* ms, int64_t* launches, double* bytes, double* flops,
                      int32_t max_n, int32_t* n_out);
/* Restricts the event pairs of the profiles that follow to the kernel classes named in `names`
 * (comma-separated, e.g. "slice_row,slice_col"; NULL or "" selects every class).  Launches of
 * the other classes are still counted, with their algorithmic bytes and flops, but get no events
 * and report 0 milliseconds, so the profile adds almost nothing to the time of unselected
 * launches.  The selection stays until the next call.  TACAW_EINVAL while a profile is being
 * recorded.  The paper has no counterpart. */
int tacaw_profile_select(tacaw_ctx* ctx, const char* names);

#ifdef __cplusplus
}
#endif
#endif /* TACAW_H */
