/*
 * tnlm.h -- C ABI of the GB300 (sm_103a) TNLM 4DCT reconstruction library.
 *
 * Method: Tian, Jia, Dong, Lou, Jiang, "Low-dose 4DCT reconstruction via
 * temporal non-local means", arXiv:1009.1351.  All N respiratory phases of
 * one slice are reconstructed together by minimising Eq. 1 with the
 * modified forward-backward splitting of Sec. 2.2:
 *
 *   repeat K times (TNLM algorithm box):
 *     g_i   = CGLS data step from f_i^(k-1)           (CGLS box; or Eq. 4)
 *     omega = Eq. 8 weights between adjacent phases from g   (Sec. 2.3 window)
 *     f     = M2 Gauss-Jacobi sweeps of Eq. 7 from g   (Gauss-Jacobi box)
 *     f     = max(f, 0)                                (positivity step)
 *
 * Conventions shared by every call
 *   - Phases are 0..N-1 (the paper's 1..N) and cyclic: f_N = f_0 (Sec. 2.1).
 *   - Images are float32 [N][ny][nx], row-major, ix fastest.  Pixel (ix, iy)
 *     has centre ((ix-(nx-1)/2)*pixel_mm, (iy-(ny-1)/2)*pixel_mm) and covers
 *     the half-open square of side pixel_mm around it.  Values are linear
 *     attenuation in 1/mm.
 *   - Sinograms are float32 [N][V][B]: phase, view, detector bin.  View v of
 *     phase i has source angle view_angles_rad[i*V + v]; the source sits at
 *     sid_mm*(cos t, sin t).  The detector is an equiangular arc centred on
 *     the source (the arc detector of Sec. 3); bin b has fan angle
 *     (b-(B-1)/2)*bin_mm/sdd_mm, counter-clockwise from the central ray.
 *   - P_i is the exact-length ray-driven projector: entry (ray, pixel) is the
 *     length in mm of the ray inside the pixel square (the quantity Siddon's
 *     method traces, Sec. 3).
 *   - Device pointers are CUDA global-memory pointers on the geometry's
 *     device, 16-byte aligned, owned by the caller; the library never frees
 *     them.  'stream' is a cudaStream_t (NULL = legacy default stream).  All
 *     calls are asynchronous on that stream unless stated otherwise.
 *   - Every call returns a tnlm_status; on failure tnlm_last_error() (per
 *     host thread) describes it.  Argument checks happen before any GPU work.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef TNLM_H
#define TNLM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TNLM_OK = 0,
    TNLM_ERR_INVALID_ARG = 1, /* a size, pointer, parameter or geometry check failed */
    TNLM_ERR_OOM = 2,         /* device workspace allocation failed (nothing leaked) */
    TNLM_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    TNLM_ERR_NUMERIC = 4,     /* a non-finite value was met in the weights or images */
    TNLM_ERR_TIMEOUT = 5      /* a bounded device-side wait (TMA pipeline of the sweep) ran out */
} tnlm_status;

enum { TNLM_DETECTOR_ARC = 0 };
enum { TNLM_DATA_CGLS = 0, TNLM_DATA_GRAD = 1 };

/* Scan geometry of one slice (Sec. 2.1: P_i maps f_i to the views of phase i). */
typedef struct {
    int nx, ny;                    /* image size in pixels, 1..8192 */
    double pixel_mm;               /* pixel side, > 0 */
    int n_phases;                  /* N in 3..4096 (with N = 2 both neighbours coincide) */
    int n_views;                   /* V >= 1 views per phase */
    int n_bins;                    /* B detector bins, 1..4096 */
    double bin_mm;                 /* bin pitch on the arc, > 0 */
    double sid_mm;                 /* source to isocentre; > image half-diagonal */
    double sdd_mm;                 /* source to detector; > sid_mm + image half-diagonal */
    int detector;                  /* TNLM_DETECTOR_ARC */
    const double* view_angles_rad; /* host [N*V] source angles, copied at creation */
    int device;                    /* CUDA device ordinal */
} tnlm_geometry_desc;

typedef struct tnlm_geometry tnlm_geometry;

/* Iteration parameters (Sec. 2.2; the paper leaves their values open). */
typedef struct {
    double mu_hat;   /* mu/beta of Eq. 7, >= 0 */
    double h;        /* kernel width of Eq. 8 (image units), > 0 */
    double beta;     /* step constant of Eq. 4 (data_step = GRAD only), > 0 */
    int patch;       /* d: odd patch side, 1..15 */
    int window;      /* W: odd search-window side, 1..31 */
    int m1;          /* CGLS steps per outer iteration, >= 0 (0: g = f^(k-1)) */
    int m2;          /* Gauss-Jacobi sweeps per outer iteration, >= 0 */
    int k_outer;     /* outer iterations K, >= 0 */
    int data_step;   /* TNLM_DATA_CGLS (CGLS box) or TNLM_DATA_GRAD (Eq. 4) */
    int clamp;       /* 1: f = max(f, 0) after each outer iteration */
    double tol;      /* > 0: stop once ||f^k - f^(k-1)|| / ||f^k|| < tol (checked on
                        the host every 'tol_check_every' iterations); 0: run K */
    int tol_check_every; /* >= 1 when tol > 0 */
    int precision;   /* TNLM_PREC_FP32: every step in FP32 (FP64 reductions);
                        TNLM_PREC_MIXED: the patch-distance cross terms of Eq. 8 as
                        split-FP16 tensor-core products with FP32 accumulation
                        (patch <= 7, window 3..15), all else as FP32 */
    int monitor;     /* 1: every outer iteration also reduces, in FP64, the TNLM term
                        of Eq. 1 (J of Eq. 2 toward both neighbours, with that
                        iteration's weights, at the iteration's result), and the call
                        ends with one more projection for the data term of the final
                        image (see tnlm_report); costs one more pass over the stored
                        distances per iteration.  0: off */
    int recompute;   /* 1: the Gauss-Jacobi sweeps recompute the Eq. 8 patch distances of
                        both directions from g^(k) in every sweep instead of reading the
                        distance array the weights step stores (that step then only forms
                        the row minima); same arithmetic, FP32 summation order may differ
                        in the last bit; FP32 only, patch <= 7, window <= 15.  0: store
                        the distances once per outer iteration and stream them (default) */
} tnlm_params;

enum { TNLM_PREC_FP32 = 0, TNLM_PREC_MIXED = 1 };

/* Host-side report of tnlm_reconstruct (all FP64 values come from FP64
 * device reductions).  Every *_hist pointer is an optional caller-owned host
 * array of k_outer entries (entry k: outer iteration k + 1) or NULL. */
typedef struct {
    int iterations;          /* outer iterations executed */
    double rel_change;       /* ||f^k - f^(k-1)||_2 / ||f^k||_2 of the last one */
    double data_residual;    /* sum_i ||Sigma^{-1/2}(P_i f_i - y_i)||^2 at the start of
                                the last outer iteration (i.e. of f^(k-1)) */
    double* rel_change_hist;
    double* residual_hist;
    long long clamped;       /* pixels the positivity step (TNLM box step 5) set to 0 in
                                the last outer iteration (0 with clamp = 0) */
    long long* clamped_hist;
    /* with params.monitor = 1 (otherwise the scalars are 0 and the arrays untouched): */
    double tnlm_term;        /* T(f^k) = sum_i [J(f_i, f_{i-1}) + J(f_i, f_{i+1})] (Eq. 2) at
                                the last result, with the last iteration's weights */
    double objective;        /* Eq. 1 at the last result: data term + (mu / 2) T, with
                                mu = mu_hat * beta (Eq. 7; with beta = 0, as the CGLS data
                                step allows, this is the data term alone) */
    double* tnlm_hist;       /* T after every iteration */
    double* data_hist;       /* data term of the image after every iteration */
    double* objective_hist;  /* Eq. 1 after every iteration */
} tnlm_report;

/* Create a geometry handle on desc->device: the fan-beam scan of Sec. 3
 * (a source on a circle, an equiangular arc detector, N phases of V views)
 * that P_i of Eq. 1 projects along.  The library copies the view angles and
 * builds its per-view / per-bin / per-ray tables on the device.
 * Errors: TNLM_ERR_INVALID_ARG (see the field comments above), TNLM_ERR_OOM,
 * TNLM_ERR_CUDA.  *out is NULL on failure. */
tnlm_status tnlm_create_geometry(const tnlm_geometry_desc* desc, tnlm_geometry** out);

/* Free the handle, its tables and its cached workspace (no counterpart in
 * the paper: resource management).  NULL is a no-op.  Synchronises the
 * handle's device. */
void tnlm_destroy_geometry(tnlm_geometry* geom);

/* d_sino[i] = P_i d_img[i] for every phase (Eq. 1).  In: image [N][ny][nx];
 * out: sinogram [N][V][B], overwritten. */
tnlm_status tnlm_project(const tnlm_geometry* geom, const float* d_img, float* d_sino,
                         void* stream);

/* Same result as tnlm_project, for callers that cannot allocate device
 * memory: code that runs while a CUDA stream capture is open, applications
 * whose device memory is fixed at start-up or fully owned by another
 * allocator, and hosts that only hand out preallocated buffers.  (This call
 * has no counterpart in the paper.)  tnlm_project keeps its layout copies in
 * the handle's workspace, which is sized for a whole reconstruction and
 * allocated on first use; this variant allocates nothing: its scratch is a
 * file-scope device array of 12 Mi floats (48 MiB) that every GPU which loads
 * the library holds until the process exits.
 *   - Limit: 2 * N * (ny * (nx + 4) + nx * (ny + 4)) floats plus alignment must
 *     fit in 12 Mi floats (e.g. 10 phases of 512 x 512); larger geometries return
 *     TNLM_ERR_INVALID_ARG and nothing is launched.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents
 *     (each call clears the part it uses before filling it).  Calls whose
 *     work overlaps on the GPU (other streams or threads) race on it.
 * Arguments, layouts and the other errors are those of tnlm_project. */
tnlm_status tnlm_project_static(const tnlm_geometry* geom, const float* d_img, float* d_sino,
                                void* stream);

/* d_img[i] = P_i^T d_sino[i] (the adjoint used by the CGLS box and Eq. 4):
 * the exact transpose of tnlm_project, computed as an atomic-free gather.
 * In: sinogram [N][V][B]; out: image [N][ny][nx], overwritten. */
tnlm_status tnlm_backproject(const tnlm_geometry* geom, const float* d_sino, float* d_img,
                             void* stream);

/* Initial image f^(0) of the TNLM algorithm box (step 1: reconstruction by
 * FBP from all projections of all N phases).  The paper does not name the
 * filter; this is equiangular fan-beam FBP: each projection is weighted by
 * sid*cos(g), convolved with the discrete ramp kernel c(0) = 1/(8 dg^2),
 * c(odd n) = -1/(2 pi^2 sin^2(n dg)), c(even n) = 0 (dg = bin_mm / sdd_mm),
 * and backprojected with weight (2 pi / (N V)) / L^2, L the source-pixel
 * distance, reading the filtered projection by linear interpolation.  It
 * assumes the N*V views cover 360 degrees evenly.
 * In: d_y [N][V][B] line integrals; out: d_img [N][ny][nx], every phase the
 * same image.  Uses the handle's workspace (allocated on first use). */
tnlm_status tnlm_fbp(const tnlm_geometry* geom, const float* d_y, float* d_img, void* stream);

/* FBP of each phase from its own V views only (the same filter, dbeta =
 * 2 pi / V): d_img[i] reconstructs phase i.  This is the per-phase FBP the
 * paper compares against (Sec. 3) and the input of the learned warm start.
 * Layout, ownership and errors as tnlm_fbp. */
tnlm_status tnlm_fbp_phases(const tnlm_geometry* geom, const float* d_y, float* d_img, void* stream);

/* Byte sizes of the two output buffers of tnlm_weights (Eq. 8 distances
 * for the W x W window of Sec. 2.3, and the per-direction normalisers). */
tnlm_status tnlm_weights_size(const tnlm_geometry* geom, const tnlm_params* params,
                              size_t* dist_bytes, size_t* norm_bytes);

/* Eq. 8 weights between every pair of adjacent phases, computed from the
 * images d_g (the CGLS output g^(k) in the algorithm).  One distance array
 * serves both directions of a pair (the symmetric reuse of Sec. 2.3):
 *
 *   d_dist [N][W*W][ny][nx]: D_i(x, s) = ||R_{g_i}(x) - R_{g_{i+1}}(x+s)||^2,
 *       the squared L2 distance of the d x d patches (values outside the
 *       image count as 0), for shift s = (sx, sy), index (sy+r)*W + (sx+r),
 *       r = (W-1)/2; +INFINITY where x+s lies outside the image.
 *   d_norm [4][N][ny][nx]: per row phase i and pixel x, the stabiliser m and
 *       the normaliser Z of each direction:
 *         [0] m_next, [1] Z_next:  omega_{i,i+1}(x, x+s) = exp(-(D_i(x,s) - m_next)/h^2) / Z_next
 *         [2] m_prev, [3] Z_prev:  omega_{i,i-1}(x, x+s) = exp(-(D_{i-1}(x+s,-s) - m_prev)/h^2) / Z_prev
 *       m is the row minimum of D, so Z >= 1, and each row sums to 1 (Eq. 3).
 * Uses the handle's cached workspace (allocated on first use). */
tnlm_status tnlm_weights(const tnlm_geometry* geom, const tnlm_params* params, const float* d_g,
                         float* d_dist, float* d_norm, void* stream);

/* Workspace the handle allocates for tnlm_reconstruct / tnlm_weights with
 * these parameters (it is cached and reused between calls; no counterpart
 * in the paper: the storage of the TNLM box's intermediate arrays). */
tnlm_status tnlm_workspace_bytes(const tnlm_geometry* geom, const tnlm_params* params,
                                 size_t* bytes);

/* The TNLM algorithm box: K outer iterations from d_f = f^(0) (for the
 * paper, the FBP of all views), result f^(K) written back into d_f.
 *   d_y    [N][V][B]  measured line integrals y_i
 *   d_winv [N][V][B]  Sigma^{-1} (diagonal inverse variance, Eq. 9), >= 0
 *   d_f    [N][ny][nx] in: f^(0), out: f^(K)
 *   rep    host report or NULL.  With rep != NULL (or tol > 0) the call
 *          synchronises the stream and checks the device numeric flag;
 *          without, it returns as soon as the work is queued and a numeric
 *          fault is reported by the next synchronising call.
 * Errors: TNLM_ERR_INVALID_ARG, TNLM_ERR_OOM, TNLM_ERR_CUDA, TNLM_ERR_NUMERIC. */
tnlm_status tnlm_reconstruct(const tnlm_geometry* geom, const tnlm_params* params,
                             const float* d_y, const float* d_winv, float* d_f,
                             tnlm_report* rep, void* stream);

/* Launch autotuner (the paper has no counterpart; it chooses how the same
 * arithmetic is laid out on the device).  Runs one outer iteration of the
 * algorithm box from d_f0 on a scratch copy (d_f0 is not modified), then
 * times the backprojection with 1..4 view groups (CTAs) per 32 x 32 tile and
 * the Gauss-Jacobi sweep with 1..3 pixel tiles per CTA under two window
 * schedules (each work unit takes the whole W x W window of its tile, or
 * the window rows in two halves as separate units whose partial sums the
 * second to finish adds), and keeps the fastest choice in the handle (used
 * by every later call on it).  Results are cached per device and shape
 * (nx, ny, N, V, B, window, patch): a second handle of the same shape is
 * tuned without timing.  The choice changes launch shapes only: the tiles
 * per CTA leave results bitwise unchanged; the number of view groups and
 * the window schedule change the order of FP32 sums (results may differ in
 * the last bits; each choice is deterministic).  Synchronises the stream;
 * allocates one image-sized scratch buffer for the duration of the call.
 * bp_groups / gj_tiles / gj_split (may be NULL) receive the choice (gj_split
 * 1: whole window, 2: two halves, 0: no sweep tuned).  Errors: as
 * tnlm_reconstruct. */
tnlm_status tnlm_autotune(tnlm_geometry* geom, const tnlm_params* params, const float* d_y,
                          const float* d_winv, const float* d_f0, int* bp_groups, int* gj_tiles,
                          int* gj_split, void* stream);

/* Batched reconstruction of many independent slices (each its own handle,
 * sizes, view counts and parameters may differ; all on one device).  Each
 * slice runs the algorithm box from d_f[i] exactly as tnlm_reconstruct
 * would, with bitwise the same result and the same stopping rule: at most
 * params[i].k_outer outer iterations, and with tol > 0 it stops at the first
 * check (every tol_check_every iterations) where the relative change is
 * below tol.  The whole run is ONE graph launch: a conditional WHILE node
 * whose body starts with a gate kernel that evaluates every slice's
 * stopping rule on the device and then runs one conditional IF node per
 * slice (that slice's outer iteration, captured once), so kernels of
 * different slices overlap and finished slices drop out without host
 * round trips.  If the runtime refuses that graph (or the environment
 * variable TNLM_BATCH_REPLAY is 1), a graph of one outer iteration of the
 * live slices is replayed instead and the stopping rules are checked on
 * the host (same results).  autotune_shapes != 0 runs
 * tnlm_autotune first on every handle not yet tuned.  reports (may be NULL)
 * is an array of count reports (iterations = that slice's own count).
 * Synchronises the stream.  Errors: as tnlm_reconstruct; the first failing
 * slice's status is returned after all reports are filled. */
tnlm_status tnlm_reconstruct_batch(tnlm_geometry* const* geoms, const tnlm_params* params,
                                   int count, const float* const* d_y, const float* const* d_winv,
                                   float* const* d_f, tnlm_report* reports, int autotune_shapes,
                                   void* stream);

/* 1 if the last tnlm_reconstruct_batch call on this host thread ran as a
 * single loop-graph launch, else 0 (no counterpart in the paper: how the
 * batched TNLM boxes were launched). */
int tnlm_batch_last_was_loop(void);

/* Kernel classes, for launch counting and optional device timing. */
enum {
    TNLM_KCLASS_PREP = 0,        /* layout copies, fills, sqrt(Sigma^{-1}) */
    TNLM_KCLASS_PROJECT = 1,     /* P (forward projection) */
    TNLM_KCLASS_BACKPROJECT = 2, /* P^T (gather backprojection) */
    TNLM_KCLASS_CGLS = 3,        /* CGLS / Eq. 4 vector updates, FP64 scalar and monitor kernels */
    TNLM_KCLASS_WEIGHTS = 4,     /* Eq. 8 patch distances, normalisers, export */
    TNLM_KCLASS_GJ = 5,          /* Gauss-Jacobi sweeps (and the M2 = 0 finalisation) */
    TNLM_KCLASS_COUNT = 6
};

/* Profiling (tracing) of the handle's kernels (no counterpart in the
 * paper; the classes are the steps of the TNLM box).  Launches of every class are
 * always counted on the host.  Classes in class_mask (bit c = class c) are
 * additionally bracketed by CUDA events recorded on the launch stream, so
 * their device time can be read back; 0 turns the timing off.  Timing adds
 * two event records per timed launch. */
tnlm_status tnlm_profile_enable(tnlm_geometry* geom, unsigned int class_mask);

/* Read the profile (no counterpart in the paper).
 * ms[TNLM_KCLASS_COUNT]: summed device time (ms) of the timed launches per
 * class; launches[TNLM_KCLASS_COUNT]: launches per class; either may be NULL.
 * Synchronises the handle's device.  reset != 0 clears both afterwards. */
tnlm_status tnlm_profile_read(tnlm_geometry* geom, double* ms, long long* launches, int reset);

/* Microbenchmarks of the device's arithmetic pipes (no counterpart in the
 * paper: they give the roofline denominators of the ALU-bound kernels).
 * fp32_ops receives the FP32 fused multiply-add rate in lane operations per
 * second (an FMA counted as one operation, as in the projector's count of
 * work per matrix entry), ex2_ops the rate of ex2.approx.f32 (the special
 * function unit the sweep's weights use); either may be NULL.  Each is the
 * best of three timed launches after a warm-up, 8 blocks of 256 threads per
 * SM with 8 independent dependency chains per thread, on a stream of its
 * own; synchronises that stream and allocates (and frees) a small output
 * buffer.  Errors: TNLM_ERR_OOM, TNLM_ERR_CUDA. */
tnlm_status tnlm_measure_peaks(int device, double* fp32_ops, double* ex2_ops);

/* Message of the last failing call on this host thread ("" if none; no
 * counterpart in the paper: error reporting). */
const char* tnlm_last_error(void);

/* Test hook for failure handling (no counterpart in the paper): the n-th
 * device allocation from now on (n >= 1) fails as if the device were out of
 * memory; n = 0 disables. */
void tnlm_debug_fail_alloc_after(int n);

/* Test hook for the timeout path (no counterpart in the paper): the
 * pipeline waits of the TMA Gauss-Jacobi sweep (Eq. 7) give up after 'polls' polls of their mbarrier (< 0:
 * the built-in limit, 2^24).  A sweep whose wait gives up stops issuing
 * copies, waits (with the built-in limit) for the copies it has in flight,
 * leaves its outputs unwritten and sets the device flag that the next
 * synchronising call reports as TNLM_ERR_TIMEOUT; the handle stays usable.
 * Affects launches issued after the call: a cached graph of an outer
 * iteration is re-captured when the limit it was captured with differs. */
void tnlm_debug_wait_limit(long polls);

#ifdef __cplusplus
}
#endif

#endif /* TNLM_H */
