/*
 * guidefill.h -- C ABI of the GB300 Guidefill shell-fill library (libguidefill.so).
 *
 * Guidefill (Hocking, MacKenzie, Schoenlieb, arxiv 1611.05319) fills an
 * inpainting domain D_h shell by shell (Algorithm 1): at step k every pixel of
 * the active boundary whose smart-order confidence exceeds c (eqs. confidence,
 * ready) gets the normalised weighted average (eq. weight) of bilinearly
 * interpolated "ghost pixels" (eq. bilinearDef) on a ball of radius eps rotated
 * to the guide direction g(x) (Notation: B~ = R(B)).  This library runs that
 * fill, the Section 3.3 guide-field construction from splines, and the adjoint
 * of the fill, as hand-written CUDA kernels for sm_103a.
 *
 * Conventions for every entry point:
 *  - All array pointers are DEVICE pointers owned by the caller, unless the
 *    name says "host".  Images are row-major [H][W] with no padding; pixel
 *    (x, y) is column x, row y, centre at integer coordinates.
 *  - Colours are float RGBA, 16-byte aligned ([H][W][4]); all four channels
 *    are filled alike.  Labels are uint8: 0 known, 1 hole (D_h),
 *    2 bystander (B_h, Section 2.1; never read, never written).
 *  - Guide fields are float [H][W][2] vectors g = (gx, gy) in pixel units
 *    along x (columns) and y (rows); only hole pixels are read.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Every call is asynchronous on that stream and never synchronises
 *    the host.  Device-side outcomes (status, shell counts) are written to a
 *    caller-owned device gf_stats array.
 *  - A call that returns GF_ERR_ARG detected the problem on the host and
 *    launched nothing.  GF_ERR_CUDA means a CUDA API call failed (the CUDA
 *    error is retrievable with gf_last_cuda_error()).
 *  - A gf_ctx owns the library's scratch memory (it grows on demand with
 *    cudaMalloc) and cached CUDA graphs; it is not thread safe: use one
 *    context per host thread / concurrent stream.
 */
#ifndef GUIDEFILL_H
#define GUIDEFILL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GF_OK = 0,
    GF_INCOMPLETE = 1,       /* some hole pixels could never be filled (walled off) */
    GF_ERR_ARG = -1,         /* invalid argument, detected on the host, nothing launched */
    GF_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    GF_ERR_TIMEOUT = -3,     /* reserved: a bounded device wait gave up */
    GF_ERR_NO_PROGRESS = -4, /* the shell loop hit max_shells before finishing */
    GF_ERR_OOM = -5,         /* scratch allocation failed */
    GF_ERR_UNSUPPORTED = -6, /* device is not sm_103 / feature unavailable */
    GF_ERR_INTERNAL = -7,    /* a device-side consistency check failed */
    GF_ERR_TOO_LARGE = -8    /* frame exceeds the fixed scratch of gf_fill_noalloc */
} gf_status;

/* gf_params.flags */
#define GF_FLAG_GHOST 1u  /* rotated ghost-pixel ball (Guidefill); off = lattice ball (coherence transport) */
#define GF_FLAG_SMART 2u  /* smart order, ready = C(x) > c (eq. ready); off = onion order */
#define GF_FLAG_RESCAN 4u /* recompute the whole active boundary every step ("without tracking", Section 3.6) */
#define GF_FLAG_DATA 8u   /* data term D(x) = |g(x)| of eq. ready2 (Section 3.5, possible extensions): while
                             some hole pixel with g != 0 is unfilled, only pixels with g != 0 are ready; eq.
                             ready from the first step at which none is left or none would be filled */

/* Opaque library context. */
typedef struct gf_ctx gf_ctx;

/*
 * One frame.  out_rgba may equal rgba (in-place fill; the fill never reads a
 * hole pixel's input colour).  out_shell receives, per pixel: -1 known,
 * -3 bystander, -2 hole pixel never filled, k >= 0 the step at which it was
 * filled.  Optional outputs (NULL to skip):
 *   out_enter [H][W] int32: step at which a hole pixel joined the active
 *             boundary (Notation, d_active D^(k)_h), -1 never / not a hole;
 *   out_stall uint32 bitmap of ceil((H*W+1)/32) words: bit k set when step k
 *             was filled by the stall rule (no front pixel was ready).
 */
typedef struct {
    int32_t H, W;
    const float *rgba;      /* [H][W][4] input colours */
    const uint8_t *labels;  /* [H][W] */
    const float *guide;     /* [H][W][2] */
    float *out_rgba;        /* [H][W][4] */
    int32_t *out_shell;     /* [H][W] */
    int32_t *out_enter;     /* [H][W] or NULL */
    uint32_t *out_stall;    /* bitmap or NULL */
} gf_frame;

/*
 * Method parameters (Section 3.2 defaults: eps = 3 px, mu = 50; Section 3.5:
 * c = 0.05).  eps in [1, 7] px (ball radius in pixels, real valued: the ball
 * is {(n,m) != 0 : n^2 + m^2 <= eps^2}); mu >= 0; c in (0, 1) for smart order;
 * snap_tau: ghost-sample offsets within snap_tau of an integer are snapped to
 * it (0 <= snap_tau < 0.01; default 1e-5); max_shells: safety cap on the
 * number of steps (0 = number of hole pixels + 1).
 */
typedef struct {
    float eps, mu, c;
    uint32_t flags;
    float snap_tau;
    int32_t max_shells;
} gf_params;

/* Per-frame device-side results. */
typedef struct {
    int32_t shells;      /* K: steps that filled at least one pixel */
    int32_t stalls;      /* steps filled by the stall rule */
    int32_t status;      /* gf_status of this frame */
    int32_t rechecks;    /* ready tests re-done in FP64 (implementation count) */
    int64_t filled;      /* hole pixels filled */
    int64_t evaluations; /* ready tests executed (implementation count) */
    int64_t max_front;   /* max over k of |d_active D^(k)_h| */
    int64_t holes;       /* |D_h| */
    int32_t data_switch; /* GF_FLAG_DATA: first step evaluated with eq. ready (-1: flag off or never) */
    int32_t reserved;
} gf_stats;

/* Creates a context bound to CUDA device `device` (must be compute capability
 * 10.3).  Returns GF_ERR_UNSUPPORTED on another device, GF_ERR_CUDA if the
 * device cannot be used. */
gf_status gf_create(gf_ctx **ctx, int device);

/* Frees the context, its scratch memory and cached graphs.  Waits for work the
 * context launched to finish.  NULL is ignored. */
void gf_destroy(gf_ctx *ctx);

/* Static string for a gf_status value. */
const char *gf_status_string(int status);

/* Last CUDA error code seen by the context (0 if none). */
int gf_last_cuda_error(const gf_ctx *ctx);

/*
 * Fills one frame (Algorithm 1 with Guidefill's ball and weights).
 * dev_stats: device pointer to one gf_stats, written when the fill ends.
 */
gf_status gf_fill(gf_ctx *ctx, const gf_frame *frame, const gf_params *params, gf_stats *dev_stats,
                  void *stream);

/*
 * gf_fill without any device allocation.  The paper has no counterpart: this
 * is for callers that cannot call cudaMalloc -- hosts that own all device
 * memory and hand libraries none, loops that must not allocate (or risk an
 * allocation failure) once they run.  The library's scratch is a fixed
 * file-scope __device__ array (about 11 MB, held by every GPU that loads the
 * library until the process exits) instead of cudaMalloc memory, so:
 *  - frames larger than 4096 x 4096 px or 4,194,304 px in total are rejected
 *    with GF_ERR_TOO_LARGE (nothing launched);
 *  - every call shares the array, which keeps the last call's contents (each
 *    call clears what must start at zero); calls that overlap on the GPU
 *    (unordered streams or host threads) race on it;
 *  - the first call on a device looks up the array's address and sets kernel
 *    attributes with that device current: make it before any stream capture;
 *    after a cudaDeviceReset of that device it must not be called again.
 * Inputs, outputs and flags (GF_FLAG_DATA included) as gf_fill; the current
 * CUDA device is used; no context.
 */
gf_status gf_fill_noalloc(const gf_frame *frame, const gf_params *params, gf_stats *dev_stats,
                          void *stream);

/*
 * Fills n independent frames in one persistent launch: each thread-block
 * cluster takes frames from a device work queue (largest hole first) and runs
 * that frame's shell loop, so frames of very different hole sizes and shell
 * counts overlap.  frames: HOST array of n descriptors; dev_stats: device
 * array of n gf_stats.  The launch sequence is captured once into a CUDA graph
 * and replayed while the descriptors and parameters stay the same.
 */
gf_status gf_fill_batched(gf_ctx *ctx, int n, const gf_frame *frames, const gf_params *params,
                          gf_stats *dev_stats, void *stream);

/*
 * gf_fill_batched that also records two caller-owned CUDA events
 * (cudaEvent_t passed as void*, NULL to skip) on `stream` immediately before
 * and after the persistent fill kernel, outside the cached graphs, so that
 * the kernel's own duration can be timed per call.  A measurement hook of
 * this implementation (no counterpart in the paper).
 */
gf_status gf_fill_batched_ex(gf_ctx *ctx, int n, const gf_frame *frames, const gf_params *params,
                             gf_stats *dev_stats, void *stream, void *event_fill_start,
                             void *event_fill_end);

/*
 * gf_fill_batched with HOST buffers (pageable or pinned): the whole step a
 * caller with frames in host memory makes.  Per frame i it copies rgba[i]
 * ([H][W][4] float), labels[i] and either guide[i] ([H][W][2] float) or, when
 * host_guide is NULL or host_guide[i] is NULL, the polylines (n_splines[i],
 * host_offsets[i], n_points[i], host_pts[i]) to device scratch owned by the
 * context; builds the guide field from the polylines if needed
 * (gf_guidance_from_splines with `eta`); fills; and copies the filled image
 * and shell map back into host_out_rgba[i] / host_out_shell[i].  host_stats:
 * n gf_stats written on the host.  Synchronises `stream` before returning.
 * In place (host_out_rgba[i] == host_rgba[i] for every frame) on host memory
 * the device can address (pinned or registered; also host_guide[i] where
 * given), only what the fill reads and writes crosses the link: the colours of
 * the 8x8 tiles within one tile of a tile holding a hole pixel (the fill reads
 * colours at most ceil(eps) + 1 <= 8 px from a hole pixel), the guide of the
 * hole tiles, and back the colours of the hole pixels, written by the device
 * into the caller's buffer; the buffer ends up as a full copy would leave it.
 */
gf_status gf_fill_batched_host(gf_ctx *ctx, int n, const int32_t *H, const int32_t *W,
                               const float *const *host_rgba, const uint8_t *const *host_labels,
                               const float *const *host_guide, const int32_t *n_splines,
                               const int32_t *const *host_offsets, const int32_t *n_points,
                               const float *const *host_pts, float eta, float *const *host_out_rgba,
                               int32_t *const *host_out_shell, const gf_params *params,
                               gf_stats *host_stats, void *stream);

/*
 * Guide field from splines (Section 3.3): for each hole pixel, the nearest
 * segment of the polylines (offsets[n_splines+1] into pts[n_points][2], (x,y)
 * pairs); if its distance d <= 3 eta, g = unit tangent * exp(-d^2/(2 eta^2)),
 * else g = 0.  The nearest segment and the 3-eta cut are decided in FP32
 * (ties: lowest segment index); the value is evaluated in FP64 and rounded once.
 * Writes guide [H][W][2] at hole pixels only.
 */
gf_status gf_guidance_from_splines(gf_ctx *ctx, int H, int W, const uint8_t *labels, int n_splines,
                                   const int32_t *offsets, int n_points, const float *pts, float eta,
                                   float *guide, void *stream);

/* One frame of a batched guide-field request. */
typedef struct {
    int32_t H, W;
    const uint8_t *labels;
    int32_t n_splines, n_points;
    const int32_t *offsets; /* device [n_splines+1] */
    const float *pts;       /* device [n_points][2] */
    float *guide;           /* device [H][W][2] */
    const float *weight;    /* device [n_splines] or NULL: |g_Gamma| of each spline (Section 3.3), the
                               factor the spline's field is multiplied by (in FP64, before the one
                               rounding); NULL = 1 */
} gf_spline_frame;

/* gf_guidance_from_splines for n frames in one launch sequence; frames is a
 * HOST array. */
gf_status gf_guidance_batched(gf_ctx *ctx, int n, const gf_spline_frame *frames, float eta,
                              void *stream);

/*
 * Guide fields from polylines and the batched fill in one call: the same results
 * as gf_guidance_batched(splines) followed by gf_fill_batched_ex(frames).  The
 * guide fields are built on the context's second stream while the fill's
 * preparation (descriptors, init pass, frame order), which does not read them,
 * runs on `stream`; the fill kernel starts once both are done.  (With
 * GF_FLAG_DATA the init pass reads the guide field, so the two run one after the
 * other.)  splines[i] must describe frame i: the same H, W, labels and guide
 * pointers.  event_fill_start / event_fill_end as in gf_fill_batched_ex.
 */
gf_status gf_fill_batched_splines(gf_ctx *ctx, int n, const gf_frame *frames, const gf_spline_frame *splines,
                                  float eta, const gf_params *params, gf_stats *dev_stats, void *stream,
                                  void *event_fill_start, void *event_fill_end);

/*
 * Automatic spline detection (Section 3.3).  A ring R of known pixels at
 * Chebyshev distance ring_dist from the hole D_h (labels == 1), with no hole or
 * bystander pixel nearer; Canny edge detection on the annulus of known pixels
 * within `annulus` of that distance; and for every ring pixel on an accepted
 * edge a straight spline of length `length` from the pixel along the minor
 * eigenvector v- of the structure tensor J_{sigma,rho} (eq. structureTensor) at
 * that pixel, signed to point into D_h, with the weight tanh((lambda+ -
 * lambda-)/Lambda) of g_Gamma.  Definitions, all in FP32 with correctly
 * rounded operations and no contraction beyond the fused multiply-adds stated:
 *  - u_sigma = g_sigma * u per colour channel (R, G, B; alpha unused); g_s has
 *    radius ceil(2 s) (window 4 s + 1), taps exp(-i^2/(2 s^2)) (FP64, rounded)
 *    divided by their FP32 sum, applied along rows then columns, taps in order
 *    -r..r, each accumulated by a fused multiply-add, image coordinates clamped;
 *  - gradient by central differences (one-sided at the border); T = sum over
 *    channels R, G, B of grad u_sigma (x) grad u_sigma, each product accumulated
 *    by a fused multiply-add; J = g_rho * T (same blur);
 *  - Canny: m2 = Txx + Tyy; direction from d = Txx - Tyy, e = 2 Txy quantised
 *    to 0/45/90/135 degrees (|e| <= d: 0; |e| <= -d: 90; e > 0: 45; else 135);
 *    kept by suppression when m2 >= m2 of both neighbours along it; strong when
 *    m2 > t_high^2, weak when m2 > t_low^2; weak pixels kept when 8-connected
 *    through kept annulus pixels to a strong one;
 *  - eigenvectors: r = sqrt(d^2 + e^2) = lambda+ - lambda- of J; v+ ~ (d + r, e)
 *    if d >= 0 else (e, r - d) ((1, 0) if both vanish), normalised, v- =
 *    (-v+_y, v+_x);
 *  - sign: -v- when the hole distance at base - ring_dist v- (rounded to the
 *    nearest pixel, clamped) is smaller than at base + ring_dist v-, else +v-;
 *  - weight = tanh(r / Lambda) in FP64, rounded.
 * Every set (ring, annulus, edges, splines) and every spline end point is
 * therefore decided by correctly rounded operations only.
 */
typedef struct {
    float sigma, rho;   /* Gaussian scales of J_{sigma,rho}; 0 < sigma <= 4, 0 < rho <= 8 */
    int32_t ring_dist;  /* dR >= 1; 0 = ceil(2 sigma) + ceil(2 rho) + 2, the smallest distance at
                           which the tensor's windows and the gradient stencil miss D_h u B_h */
    int32_t annulus;    /* 0 <= annulus <= 16, annulus < dR; ring_dist + annulus <= 96 */
    float t_high, t_low; /* Canny thresholds on |grad u_sigma| (channels in quadrature) */
    float length;       /* spline length in pixels, > 0 */
    float Lambda;       /* > 0; Section 3.3 default 1e-5 */
} gf_detect_params;

/* One frame of a detection request (all DEVICE pointers). */
typedef struct {
    int32_t H, W;
    const float *rgba;      /* [H][W][4] */
    const uint8_t *labels;  /* [H][W] */
    int32_t max_splines;    /* capacity of the outputs below, >= 0 */
    float *pts;             /* [max_splines][2][2]: base (x, y), end (x, y); 8-byte aligned */
    float *weight;          /* [max_splines] */
    int32_t *offsets;       /* [max_splines + 1]: offsets[s] = 2 min(s, n), so (pts, offsets) with
                               n_splines = max_splines, n_points = 2 max_splines is a valid input of
                               gf_guidance_batched whatever n is */
    int32_t *base;          /* [max_splines] or NULL: pixel index y W + x of each spline's base */
    uint8_t *edges;         /* [H][W] or NULL: 1 where the annulus holds an accepted edge, else 0 */
    int32_t *result;        /* [2]: result[0] = n, the number of splines found (the first
                               min(n, max_splines) in raster order of their base are written);
                               result[1] = 0, or GF_ERR_TIMEOUT if a bounded device loop gave up */
} gf_detect_frame;

/* Detection for n frames in one launch sequence (frames: HOST array).  Scratch
 * is about 28 bytes per pixel, owned by the context.  GF_ERR_ARG when a
 * parameter is out of the ranges above or a pointer is missing or misaligned. */
gf_status gf_detect_splines_batched(gf_ctx *ctx, int n, const gf_detect_frame *frames,
                                    const gf_detect_params *params, void *stream);
gf_status gf_detect_splines(gf_ctx *ctx, const gf_detect_frame *frame, const gf_detect_params *params,
                            void *stream);

/*
 * Guide field from an angle field: g = mag * (cos phi, sin phi) at hole pixels
 * (labels == 1), evaluated in FP64 and rounded once to FP32; other pixels are
 * not written.  mag, phi: [H][W] float (phi in radians, x towards columns,
 * y towards rows).  The parametrisation in which gf_fill_backward reports the
 * angle gradient.
 */
gf_status gf_guide_from_angle(gf_ctx *ctx, int H, int W, const uint8_t *labels, const float *mag,
                              const float *phi, float *guide, void *stream);

/* One frame of an adjoint request (all DEVICE pointers). */
typedef struct {
    int32_t H, W;
    const float *out_rgba;   /* [H][W][4] the forward's output */
    const float *guide;      /* [H][W][2] the forward's guide field */
    const int32_t *shell;    /* [H][W] the forward's shell map */
    const uint32_t *stall;   /* the forward's stall bitmap, or NULL if it had none */
    const float *grad_out;   /* [H][W][4] dL / d out_rgba */
    float *grad_in;          /* [H][W][4] dL / d rgba (may equal grad_out) */
    float *grad_phi;         /* [H][W] dL / d(angle of g) at fixed |g|; 0 where g = 0,
                                at stall-filled and at unfilled pixels */
    float *grad_mu;          /* one float: this frame's dL / d mu (overwritten) */
} gf_adjoint_frame;

/*
 * Adjoint of gf_fill / gf_fill_batched (reverse sweep over the steps of
 * Algorithm 1, K-1 .. 0), for the rotated ghost-pixel ball (GF_FLAG_GHOST;
 * otherwise GF_ERR_UNSUPPORTED).  The fill is differentiated as a map of the
 * known colours, the guidance angle field and mu with the shell schedule, the
 * stall steps and each sample's set of bilinear taps held fixed (piecewise
 * constant, derivative zero almost everywhere).  The forward's shell map
 * reconstructs every D^(k); no other forward state is needed.  params must be
 * those of the forward call.  grad_in is zero at filled hole pixels (their
 * input colour is never read) and equals grad_out at every other pixel plus
 * the contributions of the fills that read it.  Scatters use float atomics,
 * so the summation order (and the last bits) may vary between runs.
 * frames: HOST array of n descriptors.
 */
gf_status gf_fill_backward(gf_ctx *ctx, int n, const gf_adjoint_frame *frames, const gf_params *params,
                           void *stream);

/*
 * Launch shape of the persistent fill (no counterpart in the paper; a tuning
 * knob of this implementation).  cluster_size in {0 (automatic), 1, 2, 4, 8,
 * 16} CTAs per frame; n_clusters = number of persistent clusters (0 = as many
 * as fit, capped at the number of frames); use_graph = capture the batched
 * launch sequence into a CUDA graph and replay it (streams other than the
 * legacy default stream only).  Results do not depend on the launch shape.
 */
gf_status gf_set_launch_config(gf_ctx *ctx, int cluster_size, int n_clusters, int use_graph);

/*
 * Split schedule of the batched fill (no counterpart in the paper; a tuning knob
 * of this implementation).  The frames are taken largest hole first; with
 * split_m > 0 the first split_m of them go to a second persistent launch of
 * n_clusters clusters of cluster_size CTAs (1, 2, 4, 8 or 16), which runs beside
 * the launch set by gf_set_launch_config on the SMs it leaves free.  Frames with
 * long shell chains then get more CTAs each.  split_m = 0 turns the split off.
 * A split that does not fit (too few frames or SMs) falls back to one launch.
 * Results do not depend on the schedule.
 */
gf_status gf_set_split(gf_ctx *ctx, int split_m, int cluster_size, int n_clusters);

/* Split schedule used by the last fill call (all zero: one launch). */
gf_status gf_get_last_split(const gf_ctx *ctx, int *split_m, int *cluster_size, int *n_clusters);

/*
 * Autotuner (no counterpart in the paper): fills these frames under every
 * schedulable cluster size (1, 2, 4, 8, 16 CTAs per frame, as many persistent
 * clusters as fit), then under split schedules (the m = 1..8, 10, 12, 14, 16,
 * 20, 24 largest holes on m, 3m/4 or m/2 clusters of 8 or 16 CTAs beside the
 * best uniform launch, then split sizes and cluster counts within 2 of the best
 * split), `trials` timed runs each (CUDA events around the fill; about a hundred
 * schedules in all), and records the fastest
 * schedule in the context for later automatic fills of frames with the same
 * sizes, count, flags and ceil(eps).  The frames are filled by every trial.
 * Synchronises `stream`.  Optional outputs: the chosen cluster size of the main
 * launch and the mean fill time in ms.
 */
gf_status gf_autotune(gf_ctx *ctx, int n, const gf_frame *frames, const gf_params *params,
                      gf_stats *dev_stats, void *stream, int trials, int *best_cluster_size,
                      float *best_ms);

/* Launch shape chosen by the last fill call on this context. */
gf_status gf_get_last_launch(const gf_ctx *ctx, int *cluster_size, int *n_clusters);

/* Number of clusters of `cluster_size` CTAs that can be resident at once for
 * a fill with this eps (0 if the size cannot be launched; -1 on bad ctx). */
int gf_max_active_clusters(gf_ctx *ctx, float eps, int cluster_size);

#ifdef __cplusplus
}
#endif

#endif /* GUIDEFILL_H */
