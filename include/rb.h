/*
 * rb.h -- C ABI of the GB300 relative-binning (RB) likelihood library (librb).
 *
 * The library evaluates, for thousands of sampler walkers at once, the
 * relative-binning approximation of the Gaussian gravitational-wave
 * log-likelihood of arXiv:2404.11397 (Jim for binary neutron stars):
 *
 *   log L(theta) = sum_d [ <d_d|h_d(theta)> - <h_d(theta)|h_d(theta)>/2 ]      (Eq. 2, constant -<d|d>/2 dropped)
 *   <a|b> = 4 Re int a(f) b*(f) / S_n(f) df                                    (Eq. 3, as a sum on the grid f_k = k/T)
 *   r(f) = h(f; theta) / h(f; theta_ref) ~ r0(b) + r1(b) (f - f_m(b)) in bin b  (Eqs. 4-5, Sec. II.C)
 *   <d|h> ~ Re sum_b [A0 r0* + A1 r1*],  <h|h> ~ sum_b [B0 |r0|^2 + 2 B1 Re(r0 r1*)]
 *
 * with TaylorF2 + tidal waveforms (Sec. II.B) projected onto 1-3 detectors.
 * All compute runs in the library's own CUDA kernels for sm_103a; there is
 * no CPU fallback.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * Parameter vector theta (13 doubles, this order; Table III of the paper):
 *   0 Mc [Msun, detector-frame chirp mass]   1 q = m2/m1 in (0,1]
 *   2 chi1  3 chi2 (aligned spins)            4 Lambda1  5 Lambda2
 *   6 d_L [Mpc]  7 t_c [s, relative to the event]  8 phi_c  9 iota
 *   10 psi  11 ra  12 dec  [rad]
 * Gradients are with respect to these 13 entries (iota and dec, not cos iota
 * or sin dec; that chain rule is the caller's).
 * Unphysical walkers (q outside (0,1], Mc <= 0, d_L <= 0, any NaN/Inf) get
 * log L = -inf and a zero gradient; no error is raised for them.
 *
 * Ownership: the caller owns every theta/output buffer; an rb_event_t owns
 * its device memory until rb_event_free.  Batch calls are asynchronous and
 * stream-ordered: outputs are valid once the given stream has been
 * synchronised.  A NULL stream means the legacy default stream.
 *
 * Errors: every entry point returns an int status (RB_OK = 0 or a negative
 * RB_E* code, RB_PENDING for a poll that is not done).  rb_last_error()
 * returns a thread-local description of the most recent failure on the
 * calling thread.  No C++ exception crosses the ABI.
 */
#ifndef RB_H_
#define RB_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RB_API __attribute__((visibility("default")))
#else
#define RB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RB_OK 0
#define RB_PENDING 1        /* rb_poll: request not finished yet */
#define RB_EINVAL (-1)      /* bad argument or descriptor */
#define RB_ENOMEM (-2)      /* device or host allocation failed */
#define RB_ECUDA (-3)       /* a CUDA call failed (detail in rb_last_error) */
#define RB_ETIMEDOUT (-4)   /* rb_poll: timeout elapsed */
#define RB_EBUSY (-5)       /* rb_submit: admission refused (queue full) */
#define RB_ENOTFOUND (-6)   /* unknown ticket */
#define RB_ECLOSED (-7)     /* server shut down */

/* ---- bin placement (rb_event_desc.bin_scheme) ------------------------------ */
#define RB_BINS_PN 0        /* PN phase-bound ansatz (Sec. II.C) */
#define RB_BINS_AGNOSTIC 1  /* the waveform model's own phase directions (no PN ansatz) */

/* ---- evaluation modes ---------------------------------------------------- */
#define RB_MIXED 0          /* phase in float-float (FP32 pairs), trig/ratio/contraction FP32, sums FP64 */
#define RB_FP64 1           /* everything in native FP64 (comparison path) */
#define RB_MIXED_F64PHASE 2 /* phase accumulated in native FP64, rest as RB_MIXED */
/* RB_MIXED sums each walker's phase from FP32 pairs with exact high parts
 * scaled to the walker's largest phase term |dc_k g_k(f)|, |dtau_d f| over the
 * band.  A walker with such a term beyond 2^18 turns (~1.6e6 rad: far outside
 * where relative binning holds, the ratio to the fiducial waveform then
 * oscillating within bins) is not evaluated: its log L and gradient are NaN
 * (and the MALA step rejects it).  RB_FP64 and RB_MIXED_F64PHASE have no such
 * limit. */

#define RB_NPAR 13
#define RB_MAX_DET 3

typedef struct rb_event_s* rb_event_t;
typedef struct rb_server_s* rb_server_t;

/* One detector.  Site geometry: latitude and longitude [rad], elevation above
 * the WGS-84 ellipsoid [m], x- and y-arm azimuths [rad, clockwise from North];
 * arms have zero tilt.  data: complex128 strain on the grid, [n_freq][2]
 * (re, im).  psd: one-sided S_n(f) on the grid, [n_freq].  Both are host
 * pointers unless rb_event_desc.data_on_device is 1. */
typedef struct {
  double lat, lon, elev_m, xarm_az, yarm_az;
  const double* data;
  const double* psd;
} rb_detector_desc;

/* One event.  The grid is f_k = k / T for k = ceil(f_low T) .. floor(f_high T)
 * (both ends included), n_freq points, delta f = 1/T.  n_bins in [1, n_freq-1].
 * gmst: Greenwich sidereal angle of the event [rad].  theta_ref: fiducial
 * parameters of the relative-binning scheme (Sec. II.C, "Reference
 * parameters"). */
typedef struct {
  int32_t n_det;
  int32_t n_bins;
  rb_detector_desc det[RB_MAX_DET];
  double T, f_low, f_high, gmst;
  int32_t data_on_device;
  int32_t bin_scheme; /* RB_BINS_PN (0) or RB_BINS_AGNOSTIC */
  void* cuda_stream; /* cudaStream_t used for the build; NULL = default stream */
  double theta_ref[RB_NPAR];
} rb_event_desc;

typedef struct {
  int32_t n_det, n_bins;
  int64_t kmin, n_freq;
  double T, gmst;
  double base_logl;       /* log L_RB(theta_ref) = sum_d Re sum_b A0 - B0/2 (FP64) */
  size_t device_bytes;    /* device memory held by the event */
  double theta_ref[RB_NPAR]; /* the current fiducial parameters */
  int32_t bin_scheme;     /* the placement the edges were built with */
  int32_t reserved;
  double epsilon;         /* the placement measure's range over the band / n_bins [rad] */
} rb_event_info;

/* Build an event: grid, bin edges, fiducial waveform h0 on the full grid,
 * summary data A0, A1, B0, B1 per (detector, bin) in FP64, and the
 * device-resident edge and bin tables used by the batch calls.
 *
 * Bin placement, RB_BINS_PN (Sec. II.C; Zackay et al. 2018): B+1 edges equally
 * spaced in the PN phase bound 2 pi sum_g sgn(g) (f/f*_g)^g,
 * g in {-5/3,-2/3,1,5/3,7/3}, inverted by linear interpolation on the grid,
 * snapped to the nearest grid point, then made strictly increasing.
 * RB_BINS_AGNOSTIC (the outlook of Sec. V: bins without prior assumptions on
 * the waveform): the same placement in the measure
 * M(f) = 2 pi sum_j V_j(f) / V_j(f_high), V_j the total variation over the
 * grid of the model's phase direction dPsi(f; theta_ref)/dtheta_j for
 * j = Mc, q, chi1, chi2, Lambda1, Lambda2, t_c (directions without variation
 * left out); the edges stay fixed when a rebuild changes theta_ref.
 * epsilon = (range of the measure) / B is reported by rb_event_get_info.
 * Bin b holds grid points edges[b] <= k < edges[b+1]; the last bin also holds edges[B].
 * Summary data: A0 = 4 df sum_b d conj(h0) / S, A1 = same times (f - f_m(b)),
 * B0 = 4 df sum_b |h0|^2 / S, B1 = same times (f - f_m(b)), f_m = edge midpoint.
 *
 * The inputs are copied; the caller may free them after return (the call
 * synchronises desc->cuda_stream).  Errors: RB_EINVAL (n_det not in 1..3,
 * n_bins out of range, T or band invalid, NULL pointers, unphysical
 * theta_ref, unknown bin_scheme), RB_ENOMEM, RB_ECUDA. */
RB_API int rb_build_summary(const rb_event_desc* desc, rb_event_t* out);

/* Release an event's device memory.  The caller must make sure no batch call
 * using the event is still in flight.  NULL is accepted. */
RB_API int rb_event_free(rb_event_t ev);

/* Recompute an existing event in place for new data and/or a new fiducial
 * point -- e.g. after a reference-parameter search (Sec. II.C, "Reference
 * parameters") -- keeping its grid and bin edges: fiducial waveform h0 on the
 * full grid, summary data, tables and log L(theta_ref).  theta_ref_host: new
 * theta_ref [13] or NULL to keep it.  data[d] ([n_freq][2]) / psd[d]
 * ([n_freq]) for d < n_det, or both NULL to reuse the event's resident copy;
 * with data_on_device = 1 they are device pointers read in place (no copy,
 * they must stay valid until the stream reaches the rebuild), otherwise host
 * pointers copied into the event.  mode RB_FP64: the summary sums are formed
 * in FP64 (as rb_build_summary does).  The FP64 build that generates h0 keeps
 * it (16 B per point and detector, counted in device_bytes); later FP64 builds
 * with the same theta_ref stream the strain, the PSD and that stored h0
 * instead of regenerating it (the same sums in another order, within FP64
 * rounding), and a theta_ref argument discards it.  RB_MIXED / RB_MIXED_F64PHASE: the
 * fiducial phase is expanded in a Taylor series per 32-point chunk of the
 * grid (coefficients in FP64) and every grid point is evaluated in FP32 and
 * float-pair arithmetic, which keeps the per-point work off the FP64 pipe
 * (used when T f_low >= 1024 and N <= 2^30, otherwise the FP64 sums are used).
 * Asynchronous on `stream`, allocates nothing; batch calls ordered after it
 * on the same stream see the new tables, and the caller must not run batches
 * of this event concurrently on other streams.  Errors: RB_EINVAL (NULL
 * event, only one of data/psd, unphysical theta_ref, bad mode), RB_ECUDA. */
RB_API int rb_event_rebuild(rb_event_t ev, const double* theta_ref_host, const double* const* data,
                            const double* const* psd, int data_on_device, int mode, void* stream);

RB_API int rb_event_get_info(rb_event_t ev, rb_event_info* info);

/* Copy the event's FP64 summary data (A0, A1, B0, B1 of Sec. II.C, per
 * detector and bin) and bin edges to host buffers:
 * A0, A1: [n_det][n_bins][2]; B0, B1: [n_det][n_bins]; edges: [n_bins+1]
 * grid indices (0 .. n_freq-1).  Any pointer may be NULL.  Synchronous. */
RB_API int rb_event_get_summary(rb_event_t ev, double* A0, double* A1, double* B0, double* B1, int64_t* edges);

/* Checkpoint and resume an event.  rb_event_save writes to `path` everything
 * that defines the event: the descriptor (sites, T, band, gmst, n_bins), the
 * current theta_ref, and the resident FP64 strain [n_det][n_freq][2] and PSD
 * [n_det][n_freq], behind a fixed header (native byte order).  It first
 * synchronises the device, so that calls already issued on any stream are
 * included.  rb_event_load reads such a file and builds a new event from it
 * with rb_build_summary (host data, `stream` as the build stream, synchronous).
 * The build is deterministic, so the loaded event's grid, bins, summary data,
 * tables and log L values are bit-identical to those of an event built from
 * the same inputs.  Errors: RB_EINVAL (NULL argument, unreadable or unwritable
 * path, a file that is not a complete event file, or an event whose last
 * rebuild read caller data in place: it holds no copy of that data);
 * rb_build_summary's errors on load; RB_ECUDA. */
RB_API int rb_event_save(rb_event_t ev, const char* path);
RB_API int rb_event_load(const char* path, void* stream, rb_event_t* out);

/* Batched RB log-likelihood: the network likelihood of Sec. II.A (Eqs. 2-3)
 * in its relative-binning form (Sec. II.C, Eqs. 4-5), the waveform ratio to
 * the fiducial waveform linear within each bin and contracted with the
 * summary data.  theta_dev: device [W][13] row-major FP64;
 * logl_dev: device [W] FP64.  mode: RB_MIXED, RB_FP64 or RB_MIXED_F64PHASE.
 * Asynchronous on `stream` (cudaStream_t).  W = 0 is a no-op.
 * Errors: RB_EINVAL (NULL event/pointers with W > 0, W < 0, bad mode),
 * RB_ENOMEM (stream-ordered workspace allocation), RB_ECUDA. */
RB_API int rb_loglike_batch(rb_event_t ev, const double* theta_dev, int64_t W, double* logl_dev, int mode,
                     void* stream);

/* Batched RB log-likelihood (as rb_loglike_batch, Sec. II.C) and its
 * gradient -- the gradient the MALA local sampler of Sec. II.D needs -- with respect to the 13
 * parameters (hand-written reverse sweep over bins and edges, then the chain
 * rule through the per-walker set-up).  grad_dev: device [W][13] FP64.
 * Same conventions and errors as rb_loglike_batch. */
RB_API int rb_loglike_grad_batch(rb_event_t ev, const double* theta_dev, int64_t W, double* logl_dev, double* grad_dev,
                          int mode, void* stream);

/* rb_event_rebuild (the summary data of Sec. II.C) from the event's resident data and current theta_ref
 * followed by rb_loglike_grad_batch, in one call (grad_dev may be NULL for
 * log L only): the results are those of the two calls in sequence on
 * `stream`.  With RB_MIXED and the chunk-expanded summary (T f_low >= 1024,
 * n_freq <= 2^30) the walkers' set-up, which needs only the reference values
 * and theta, runs on the event's forked stream concurrently with the summary
 * sums and is joined before the likelihood kernel; otherwise the two calls
 * run in sequence.  theta_dev must be ready on `stream` when the call is
 * made.  Asynchronous.  The per-walker workspace is kept by the event between
 * calls: it is allocated (cudaMalloc) when a call needs more than the event
 * holds and the stream is not being captured; a call captured in a graph
 * with a larger batch than any before it takes its workspace from the
 * stream-ordered pool instead.  Outgrown workspaces are released with the
 * event, so graphs that captured them stay valid while the event lives.  The
 * event's auxiliary stream for the tangents is created by its first combined
 * call, which should therefore not be inside a global-mode stream capture.
 * Errors: those of the two calls. */
RB_API int rb_rebuild_loglike_grad(rb_event_t ev, const double* theta_dev, int64_t W, double* logl_dev,
                                   double* grad_dev, int mode, void* stream);

/* End-to-end form of rb_rebuild_loglike_grad (summary data, log L and
 * gradient of Sec. II.C) for host buffers: brings the
 * new strain data_host[d] ([n_freq][2]) and PSD psd_host[d] ([n_freq]) of
 * every detector into the event's resident copy and theta_host [W][13] to
 * the device, rebuilds the summary data (current theta_ref), evaluates log L
 * (and the gradient unless grad_host is NULL), copies logl_host [W] (and
 * grad_host [W][13]) back and synchronises `stream`.  The strain and PSD
 * move on the event's copy stream while the kernels that do not read them
 * (reference values, walker set-up) run.  Pinned (page-locked, mapped)
 * buffers whose data_host[d] start on a 16-byte and psd_host[d] on an 8-byte
 * boundary are read by one kernel over the host link, which writes the
 * resident FP64 copy and the FP32 working copy in the same pass; other
 * buffers are copied by the copy engine and then converted.  Both give the
 * same bits.  When logl_host (and grad_host, if not NULL) are pinned, mapped
 * buffers starting on 8-byte boundaries, the likelihood kernel writes them
 * directly and no copy back is made.  When every buffer is pinned and mapped
 * (theta_host too, read by the set-up kernel over the host link), the call's
 * launches are captured as a CUDA graph the first time for these buffers, W
 * and mode, and replayed by the following calls with the same ones (the
 * graph reads whatever the buffers hold at each call; a call with other
 * buffers captures anew; the graph lives as long as the event; calls on one
 * event from several host threads are serialised for the capture).  Not
 * with trace events set (rb_set_trace_events).  Results equal rb_event_rebuild
 * with the same host data followed by rb_loglike_grad_host.  Errors: those of
 * the two calls. */
RB_API int rb_rebuild_loglike_grad_host(rb_event_t ev, const double* const* data_host, const double* const* psd_host,
                                        const double* theta_host, int64_t W, double* logl_host, double* grad_host,
                                        int mode, void* stream);

/* End-to-end convenience form of rb_loglike_grad_batch (Sec. II.C log L and
 * its gradient) for host buffers:
 * copies theta_host [W][13] to the device, evaluates, copies logl_host [W]
 * (and grad_host [W][13] unless NULL) back, and synchronises the stream.
 * pinned, mapped, 8-byte-aligned theta_host is read by the set-up kernel
 * over the host link (no copy in), and such logl_host/grad_host are written
 * by the likelihood kernel directly (no copy back).  With all three pinned,
 * the set-up and likelihood launches are captured as a CUDA graph the first
 * time for these buffers, W and mode, and replayed by the following calls
 * with the same ones (as for rb_rebuild_loglike_grad_host). */
RB_API int rb_loglike_grad_host(rb_event_t ev, const double* theta_host, int64_t W, double* logl_host, double* grad_host,
                         int mode, void* stream);

/* MALA local step (Sec. II.D: the sampler's local proposal is the
 * Metropolis-adjusted Langevin algorithm) for W chains, fused with the
 * likelihood and its adjoint.  Chains live in the sampling coordinates of
 * Table II, z = (Mc, q, chi1, chi2, Lambda1, Lambda2, d_L, t_c, phi_c,
 * cos iota, psi, ra, sin dec), row-major [W][13] FP64 on the device, with the
 * uniform prior of Table II on the open box lo < z < hi (host arrays of 13;
 * the cos iota and sin dec bounds must lie in [-1, 1]): log pi(z) =
 * log L(theta(z)) inside (the prior constant is dropped), -inf outside.
 *
 * rb_mala_init: logp_dev [W] = log pi(z), gz_dev [W][13] = d log pi / dz.
 * rb_mala_step: with step sizes eps_host[13], standard normal draws xi_dev
 *   [W][13] and uniform draws u_dev [W] in (0, 1] (both on the device, drawn by
 *   the caller), proposes z' = z + eps^2/2 gz + eps xi, evaluates log pi(z')
 *   and its gradient, and accepts when log u < log alpha with
 *     log alpha = log pi(z') - log pi(z) - 1/2 sum_j [(xi_j + eps_j (gz_j + gz'_j)/2)^2 - xi_j^2];
 *   z_dev, logp_dev and gz_dev are updated in place for accepted chains and
 *   accepted_dev [W] (int, may be NULL) is set to 1/0.
 * mode: RB_MIXED, RB_FP64 or RB_MIXED_F64PHASE (as rb_loglike_grad_batch).
 * Asynchronous on `stream`; per call a workspace of ~240 B + the batch's per
 * chain comes from the stream-ordered pool.  Errors: RB_EINVAL (NULL
 * pointers, bad mode, empty box, negative step size), RB_ENOMEM, RB_ECUDA. */
RB_API int rb_mala_init(rb_event_t ev, const double* z_dev, int64_t W, const double* lo_host, const double* hi_host,
                        double* logp_dev, double* gz_dev, int mode, void* stream);
RB_API int rb_mala_step(rb_event_t ev, double* z_dev, double* logp_dev, double* gz_dev, int64_t W,
                        const double* eps_host, const double* lo_host, const double* hi_host, const double* xi_dev,
                        const double* u_dev, int* accepted_dev, int mode, void* stream);

/* Full (un-binned) log-likelihood of Eq. 2 with the inner product of Eq. 3
 * on the event's whole frequency grid, for W walkers: the quantity relative
 * binning approximates (Sec. II.C), used to search for the reference
 * parameters and to measure the binning error.  The constant -<d|d>/2 is
 * dropped, as in rb_loglike_batch.  theta_dev: device [W][13] FP64;
 * logl_dev: device [W] FP64, -inf for an unphysical walker.  The data are the
 * ones the event's last rebuild summed over; <h|h> per detector is
 * |K_d(theta)|^2 sum_b B0_{d,b} / |K_d(theta_ref)|^2 (Newtonian amplitude,
 * exact), <d|h> is a sum over every grid point with the walker's phase
 * expanded per 32-point chunk (FP32 / float-pair arithmetic, FP64 sums).
 * mode: RB_MIXED only.  Needs T f_low >= 1024 and n_freq <= 2^30 (the chunk
 * expansion), and, if the last rebuild read caller data in place in RB_FP64
 * mode, a rebuild in a mixed mode or from resident data first.  Asynchronous
 * on `stream`; a workspace of 224 B per walker comes from the stream-ordered
 * pool.  Errors: RB_EINVAL (NULL pointers, W < 0, bad mode, grid outside the
 * expansion's range, data not available), RB_ENOMEM, RB_ECUDA. */
RB_API int rb_loglike_full_batch(rb_event_t ev, const double* theta_dev, int64_t W, double* logl_dev, int mode,
                                 void* stream);

/* Allocation-free form of rb_loglike_grad_batch (the paper has no
 * counterpart: it is an interface for callers that cannot allocate device
 * memory at call time -- e.g. a host framework whose own allocator owns all
 * device memory and forbids other allocations, or a latency-critical sampler
 * loop that must not pay for, or synchronise on, an allocation).  Same arguments,
 * results and errors as rb_loglike_grad_batch (grad_dev may be NULL for log L
 * only), but the per-walker workspace is a fixed device array inside the
 * library (RB_STATIC_MAX_WALKERS records, about 7.5 MiB, held on every device
 * that loads the library until exit), so the call allocates nothing.
 * W > RB_STATIC_MAX_WALKERS returns RB_EINVAL.  The first call on a device
 * looks up the array's address (cudaGetSymbolAddress) and should come before
 * any stream capture.  All calls share the array: calls whose kernels can
 * overlap on the GPU race and must be ordered by the caller.  Asynchronous on
 * `stream`. */
#define RB_STATIC_MAX_WALKERS 8192
RB_API int rb_loglike_grad_batch_static(rb_event_t ev, const double* theta_dev, int64_t W, double* logl_dev,
                                        double* grad_dev, int mode, void* stream);

/* TaylorF2 + tidal detector strain h_d(f; theta) (FP64; the waveform model
 * of Sec. II.B, projected onto the detector as in Sec. II.A) on the grid
 * f_k = (kmin + k)/T, k = 0..n_freq-1, for one source: geom = {lat, lon,
 * elev_m, xarm_az, yarm_az}, theta_host [13].  h_dev: device [n_freq][2].
 * Asynchronous on `stream`.  Used to inject signals and as the fiducial
 * waveform kernel of rb_build_summary.  Errors: RB_EINVAL, RB_ECUDA. */
RB_API int rb_strain(const double* geom, double gmst, const double* theta_host, double T, int64_t kmin, int64_t n_freq,
              double* h_dev, void* stream);

/* ---- serving loop (continuous batching) ----------------------------------
 * A server owns a scheduler thread, a set of CUDA streams ("slots") and
 * pinned staging buffers.  Clients submit likelihood(+gradient) requests for
 * resident events from any thread; requests that arrive while others are on
 * the GPU are admitted as soon as a slot and enough of the device-memory
 * budget are free, and run concurrently on separate streams.  When a slot
 * frees up, the scheduler takes the oldest pending request and packs into
 * the same launch the later pending requests for the same event and
 * gradient flag, up to max_walkers walkers and the memory budget; the
 * launch runs the packed walkers rounded up to a multiple of 256 (the extra
 * walkers are copies of the first, their results dropped), and each request
 * gets its own walkers' results back.  A launch is a CUDA graph: copy-in,
 * set-up, likelihood kernel, copy-out and a completion node, captured for the
 * launch and applied to the slot's instantiated graph for the same detector
 * count and gradient flag (cudaGraphExecUpdate; a new instantiation only when
 * the update is refused).  Results are returned by rb_poll; each is
 * identical to the same request evaluated alone (one warp per walker, no
 * cross-walker arithmetic). */
typedef struct {
  size_t hbm_budget_bytes;  /* device bytes the in-flight requests may hold (0 = 1 GiB) */
  int32_t max_slots;        /* concurrent requests on the GPU (streams), 1..64 (0 = 8) */
  int32_t max_queue;        /* pending requests before rb_submit returns RB_EBUSY (0 = 4096) */
  int32_t use_graphs;       /* 1 = replay captured CUDA graphs (default), 0 = plain launches */
  int32_t mode;             /* RB_MIXED / RB_FP64 / RB_MIXED_F64PHASE */
  int64_t max_walkers;      /* largest request accepted, and the most walkers one launch packs (0 = 65536) */
} rb_server_opts;

typedef struct {
  uint64_t submitted, completed, rejected;
  uint64_t graph_launches, plain_launches; /* launches (each may carry several packed requests) */
  uint64_t graphs_captured;   /* graph instantiations */
  int32_t in_flight, queued;  /* launches on the GPU, requests waiting */
  size_t hbm_in_use;
  int32_t max_in_flight;      /* largest number of launches on the GPU at once so far */
  int32_t reserved;
  uint64_t graph_updates;     /* launches that updated an instantiated graph in place */
  uint64_t walkers_requested; /* walkers of the completed requests */
  uint64_t walkers_run;       /* walkers their launches ran (requested + padding) */
} rb_server_stats;

RB_API int rb_server_create(const rb_server_opts* opts, rb_server_t* out);
/* Stops the scheduler after the in-flight launches finish; pending requests
 * fail with RB_ECLOSED.  A launch whose stream reports a CUDA error fails its
 * requests (RB_ECUDA) instead of being waited for, and after 30 s without
 * completion the remaining in-flight requests fail with RB_ETIMEDOUT and their
 * slots' buffers are left allocated (never freed under a running kernel). */
RB_API int rb_server_destroy(rb_server_t srv);
/* Enqueue a request for log L (Sec. II.C) and, if want_grad, its gradient
 * for W walkers of one event: theta_host [W][13] is copied before return.  *ticket
 * identifies it for rb_poll.  RB_EBUSY if the queue is full, RB_EINVAL for
 * W < 1, W > max_walkers or a NULL event. */
RB_API int rb_submit(rb_server_t srv, rb_event_t ev, const double* theta_host, int64_t W, int want_grad,
              uint64_t* ticket);
/* Wait up to timeout_us (0 = do not wait, < 0 = wait without limit) for a
 * request; on RB_OK copies logl_out [W] and, if the request wanted it and
 * grad_out != NULL, grad_out [W][13], W being the request's own (the W given
 * to rb_submit: the caller's buffers must hold that many), and forgets the
 * ticket (on a failed request too).  Returns
 * RB_PENDING (timeout_us == 0 and not done), RB_ETIMEDOUT, RB_ENOTFOUND, or
 * the request's own error status. */
RB_API int rb_poll(rb_server_t srv, uint64_t ticket, int64_t timeout_us, double* logl_out, double* grad_out);
/* The walker count and gradient flag of a request not yet collected, so that
 * the caller can size rb_poll's buffers: RB_OK, or RB_ENOTFOUND. */
RB_API int rb_ticket_info(rb_server_t srv, uint64_t ticket, int64_t* W, int32_t* want_grad);
RB_API int rb_server_get_stats(rb_server_t srv, rb_server_stats* stats);
/* Latency of the requests completed since the last reset, measured by the
 * server: part 0 from rb_submit to the moment the results are in host memory
 * (what rb_poll then copies), and its three parts: 1 waiting for a slot (and
 * budget), 2 the host staging and issuing the launch, 3 the device work and
 * the completion node.  count, and nearest-rank p50, p99 and maximum in ms (0
 * with no requests).  reset != 0 forgets all parts afterwards.  At most 4 Mi
 * requests are kept between resets. */
RB_API int rb_server_latency(rb_server_t srv, int part, int reset, int64_t* count, double* p50_ms, double* p99_ms,
                             double* max_ms);

/* ---- diagnostics ---------------------------------------------------------- */
RB_API const char* rb_strerror(int status);
RB_API const char* rb_last_error(void);
/* Tracing: record the CUDA events before_main / after_main (cudaEvent_t, or
 * NULL to stop) on the launch stream immediately before and after the main
 * likelihood kernel of every subsequent batch call (process-wide). */
RB_API void rb_set_trace_events(void* before_main, void* after_main);
/* Number of this library's kernel launches on the calling process so far
 * (all entry points, all threads). */
RB_API uint64_t rb_kernel_launch_count(void);
RB_API int rb_abi_version(void);

/* Debug builds (compiled with -DRB_BOUNDS_CHECK, e.g. librb_checked.so): the
 * number of checked device-side indices found outside their buffers since
 * the last call -- in the likelihood kernels (walker and tangent records, the
 * edge and bin tables, shared-memory staging, the outputs) and the summary
 * kernels (parts, grid points, chunk records, staging) -- with the first
 * one's site code, index and limit (NULL pointers are skipped); the records
 * are cleared.  A checked index outside its buffer is replaced by 0, so the
 * access stays in bounds and the results are wrong but the context is not.
 * Synchronous.  Returns -1 in normal builds (no checks compiled in), RB_ECUDA
 * if the records cannot be read. */
RB_API int rb_debug_bounds(int* site, long long* index, long long* limit);

#ifdef __cplusplus
}
#endif
#endif /* RB_H_ */
