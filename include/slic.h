/*
 * slic.h -- C ABI of libslicgb.so: SLIC superpixel segmentation on one
 * NVIDIA GB300 (sm_103a), following gSLICr (Ren, Prisacariu and Reid,
 * "gSLICr: SLIC superpixels at over 250Hz", arXiv 1509.04232).
 *
 * Conventions for every call
 * --------------------------
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device,
 *    owned by the caller; the library never frees them. Pointers named h_*
 *    are host pointers. `stream` is a cudaStream_t passed as void* (NULL =
 *    the legacy default stream).
 *  - Work is enqueued on `stream` and the call returns without waiting for
 *    it, unless the description says otherwise. Buffers must stay valid
 *    until the stream reaches that work.
 *  - A handle owns its device scratch (allocated in slic_create) and is not
 *    thread-safe: use one handle per host thread and per stream.
 *  - Every call returns a slic_status. On failure slic_last_error() gives a
 *    one-line reason. CUDA launch errors map to SLIC_ERR_CUDA.
 *  - Images are 8-bit R,G,B (in_channels = 3) or R,G,B,A (in_channels = 4,
 *    alpha ignored), row-major, rows of width*in_channels bytes.
 *  - Labels are int32 [height][width]; label k = r*ns_c + c names the grid
 *    cell (column c, row r) the centre started in (except with
 *    enforce_connectivity = 2, which renumbers the segments 0, 1, ...).
 *  - Centres are float [K_eff][6] = (f0, f1, f2, x, y, count) where
 *    (f0,f1,f2) = (L*, a*, b*) for SLIC_CIELAB, K_eff = ns_c*ns_r.
 *  - Features are float [3][height][width] (planar).
 *  - The library keeps per-device state (the sRGB table, kernel attributes,
 *    fault-injection words) from its first use on a device: do not use it
 *    after cudaDeviceReset on that device.
 */
#ifndef SLIC_H
#define SLIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slic_ctx *slic_handle;

typedef enum {
    SLIC_OK = 0,
    SLIC_ERR_INVALID = -1, /* bad argument or size; nothing was enqueued */
    SLIC_ERR_NOMEM = -2,   /* device or host allocation failed */
    SLIC_ERR_CUDA = -3,    /* a CUDA call or kernel launch failed */
    SLIC_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up */
    SLIC_ERR_STATE = -5    /* call not valid in the handle's state */
} slic_status;

/* Feature space of Sec. 2 / Sec. 4 (the listing's color_space setting). */
typedef enum {
    SLIC_CIELAB = 0, /* sRGB (IEC 61966-2-1) -> CIE 1976 L*a*b*, D65 */
    SLIC_RGB = 1,    /* raw R,G,B bytes as floats */
    SLIC_XYZ = 2     /* CIE XYZ (D65) x 100 */
} slic_color_space;

/* Problem statement of Sec. 2 (K or S, m) and the settings of the Sec. 4
   listing (color_space, no_iters, do_enforce_connectivity). */
typedef struct {
    int width, height;        /* > 0 */
    int K;                    /* desired superpixel count, used when S == 0:
                                 S = max(1, round(sqrt(width*height/K))) */
    int S;                    /* grid interval in pixels; > 0 overrides K */
    float m;                  /* compactness, >= 0 (Eq. 1) */
    int iterations;           /* >= 0: centre updates after the first assignment */
    int color_space;          /* slic_color_space */
    int enforce_connectivity; /* 0: none; 1: the paper's two-pass local rule
                                 (Sec. 3); 2: the original SLIC's components
                                 (Sec. 2): 4-connected segments of equal
                                 labels, one of at most S*S/4 pixels joins
                                 the segment of its first pixel's left (in
                                 column 0: upper) neighbour, the segment of
                                 pixel 0 is kept, and the kept segments are
                                 renumbered 0, 1, ... in scan order of their
                                 first pixels (labels then no longer index
                                 the centres) */
    int in_channels;          /* 3 or 4 */
    /* Sec. 2 steps of the original SLIC that the paper's GPU steps omit
       (both off by default, i.e. zero-initialised): */
    int perturb_seeds;        /* 0 or 1: move each grid seed to the pixel of
                                 lowest gradient G = |I(x+1,y)-I(x-1,y)|^2 +
                                 |I(x,y+1)-I(x,y-1)|^2 (features; neighbours
                                 clamped at the border) in the 3x3 pixels
                                 around it; it moves only to a strictly lower
                                 G, the first in scan order (dy, then dx) */
    float convergence;        /* >= 0, finite: stop after the first iteration
                                 whose update moved the centres by a mean L1
                                 distance (|dx| + |dy| in pixels, over all
                                 K_eff centres) below this; `iterations` is
                                 then the maximum. 0: fixed iterations */
} slic_params;

/* Create a handle for one image geometry; allocates the handle's device
   scratch on the current device. Grid (Sec. 2): ns_c = ceil(width/S),
   ns_r = ceil(height/S). Returns SLIC_ERR_INVALID for bad params (also
   when K_eff exceeds 2^26 or an image exceeds 2^31 pixels). */
slic_status slic_create(const slic_params *params, slic_handle *out);

/* Release the handle and its scratch (waits for the device to finish any
   work of this handle first). NULL is accepted. */
slic_status slic_destroy(slic_handle h);

/* Grid of the handle: S, ns_c, ns_r (any may be NULL). */
slic_status slic_grid(slic_handle h, int *S, int *ns_c, int *ns_r);

/* Whole segmentation, in the order of the Sec. 4 Perform_Segmentation
   listing: colour conversion (Sec. 3 "Image space conversion"), grid
   initialisation ("Cluster center initialisation"), assignment (Eq. 1,
   "Finding the cluster associations"), `iterations` x {update ("Updating
   the cluster center"), assignment}, then two connectivity passes ("Enforce
   connectivity") when enabled.
     d_image    uint8 [height][width][in_channels]
     d_labels   int32 [height][width], output
     d_centres  float [K_eff][6], output: the centres the final labels were
                assigned against (count = members in that assignment's
                input partition; 0 for an empty cluster, which keeps its
                previous position and colour)
   When slic_set_init_centres() armed initial centres, they replace the grid
   initialisation for this call only. */
slic_status slic_segment(slic_handle h, const uint8_t *d_image, int32_t *d_labels, float *d_centres,
                         void *stream);

/* Component-based connectivity (enforce_connectivity = 2) on its own:
   d_in -> d_out label maps of the handle's size (they may be the same
   buffer). SLIC_ERR_STATE unless the handle was created with mode 2 (it
   owns the scratch: 16 bytes per pixel). */
slic_status slic_connectivity_components(slic_handle h, const int32_t *d_in, int32_t *d_out, void *stream);

/* Wait for the device, then report whether a bounded device loop of the
   handle's component connectivity gave up since the last call
   (SLIC_ERR_TIMEOUT; the labels are then incomplete). Clears the flag. */
slic_status slic_status_check(slic_handle h);

/* Wait for the device, then report how many centre updates the last
   slic_segment call performed: params.iterations, or fewer when the
   stopping test (params.convergence > 0) ended the run early. A run that
   stops skips its remaining updates and middle assignment passes; its last
   assignment pass (labels against the final centres) and connectivity
   always run. */
slic_status slic_iterations_run(slic_handle h, int *out);

/* Use d_init [K_eff][6] (e.g. the previous video frame's centres) instead of
   the grid initialisation on the next slic_segment call. The buffer is read
   when that call's work runs. Pass NULL to disarm. */
slic_status slic_set_init_centres(slic_handle h, const float *d_init);

/* Sec. 3 "Image space conversion" only: d_features float [3][height][width]. */
slic_status slic_convert(slic_handle h, const uint8_t *d_image, float *d_features, void *stream);

/* Sec. 3 "Cluster center initialisation" only, from converted features. */
slic_status slic_init_centres(slic_handle h, const float *d_features, float *d_centres, void *stream);

/* One assignment pass (Eq. 1): every pixel takes the centre with the
   smallest D_s among the (at most) nine centres of its own grid cell and
   the eight around it; exact ties go to the first in scan order (dy outer,
   dx inner). d_features float [3][H][W], d_centres float [K_eff][6],
   d_labels int32 [H][W] output. */
slic_status slic_assign(slic_handle h, const float *d_features, const float *d_centres, int32_t *d_labels,
                        void *stream);

/* One centre update (Sec. 3 "Updating the cluster center") from a label map:
   centre k = mean (f0,f1,f2,x,y) of the pixels labelled k, count = their
   number; a centre with no pixels keeps d_centres_in's values and gets
   count 0. Labels must lie in [0, K_eff) (else the result is undefined for
   those pixels; they are ignored). d_centres_in may equal d_centres_out. */
slic_status slic_update(slic_handle h, const float *d_features, const int32_t *d_labels,
                        const float *d_centres_in, float *d_centres_out, void *stream);

/* One connectivity pass (Sec. 3 "Enforce connectivity"): a pixel whose
   every in-image 4-neighbour has a different label takes the most frequent
   neighbour label (ties: earliest of left, up, right, down). Reads d_in,
   writes d_out; they must not overlap. */
slic_status slic_connectivity_pass(slic_handle h, const int32_t *d_in, int32_t *d_out, void *stream);

/* Kernel launches enqueued by this handle since creation (all calls). */
slic_status slic_launch_count(slic_handle h, long long *count);

/* Per-kernel device-time accounting, for measurement. Enabling (from the
   disabled state) forgets earlier records; while enabled, the library
   records a CUDA event pair around every assignment-kernel launch it
   enqueues, on the launching stream (inside a stream capture these become
   event-record nodes that every replay of the graph re-records).
   slic_profile_read waits for those events and returns the summed duration
   (ms) of the recorded pairs and their number; it does not reset them. */
slic_status slic_profile_enable(slic_handle h, int enable);
slic_status slic_profile_read(slic_handle h, double *assign_ms, long long *assign_launches);

/* ---- Batches: many frames in one set of launches -------------------------
   A batch segments n frames that may differ in size, S (or K), m, colour
   space and channels (iterations and connectivity are shared) with one
   launch per stage for all frames: the assignment kernel is persistent, its
   grid sized to the GPU, looping over the 32x32 tiles of every frame. Per
   frame the results are bit-identical to slic_segment's. The enqueued work
   can be captured into a CUDA graph and replayed. */
typedef struct slic_batch_ctx *slic_batch;

/* params[f] describes frame f (same rules as slic_create); all frames need
   the same iterations and enforce_connectivity, while perturb_seeds and
   convergence may differ per frame. Allocates the batch's device scratch
   (12*H*P + 48*K_eff + 4*W*H + 48*(ns_c+2)*(ns_r+2) bytes per frame plus a
   256-byte state record, 256-aligned parts). */
slic_status slic_batch_create(const slic_params *params, int n_frames, slic_batch *out);

/* Bind the frames' buffers: host arrays of n device pointers, as in
   slic_segment (d_images[f] uint8 image, d_labels[f] int32 labels,
   d_centres[f] float [K_eff_f][6] centres). d_init may be NULL, or an array
   whose entry f is NULL or a float [K_eff_f][6] set of initial centres used
   instead of the grid initialisation (e.g. the previous video frame's
   centres; d_init[f] may equal d_centres[f]). Waits for the device to be
   idle, then uploads the frame table (synchronous). */
slic_status slic_batch_set_buffers(slic_batch b, const uint8_t *const *d_images, int32_t *const *d_labels,
                                   float *const *d_centres, const float *const *d_init);

/* Bind other buffers (same arguments as slic_batch_set_buffers) without
   waiting for the device: the batch keeps two copies of its frame tables,
   and this call fills the one not in use from page-locked staging memory
   with one cudaMemcpyAsync on `stream`; slic_batch_segment calls enqueued
   afterwards use it. Work already enqueued keeps the tables it was given
   (a CUDA graph captured earlier keeps using its copy, which the rebind
   after next overwrites). Calls that use the batch must be ordered on
   `stream` (or synchronised with it). SLIC_ERR_STATE before the first
   slic_batch_set_buffers. It waits only if the staging copy it needs is
   still being uploaded from the rebind before last. */
slic_status slic_batch_rebind(slic_batch b, const uint8_t *const *d_images, int32_t *const *d_labels,
                              float *const *d_centres, const float *const *d_init, void *stream);

/* Segment every frame of the batch (Sec. 4 stage order, as slic_segment);
   SLIC_ERR_STATE before slic_batch_set_buffers. */
slic_status slic_batch_segment(slic_batch b, void *stream);

/* End to end with host buffers, on `stream`: copy each frame's image from
   host_images[f] (uint8 [H][W][C]) into the bound device image, segment as
   slic_batch_segment, then copy the bound labels and centres into
   host_labels[f] (int32 [H][W]) and host_centres[f] (float [K_eff_f][6]).
   host_labels or host_centres (or an entry of them) may be NULL to skip
   those copies. One cudaMemcpyAsync per run of frames whose buffers lie
   back to back both on the host and on the device (a batch held in one
   host and one device allocation moves with one copy per direction and
   buffer kind); host memory must be page-locked for the copies to overlap
   other work. With frame groups (slic_batch_set_groups) each group's stream
   copies the group's frames in, segments them and copies its results out,
   so one group's copies overlap the other groups' kernels; the streams are
   forked from and joined back to `stream`. Returns once everything is
   enqueued: synchronise the stream before reading the outputs. Two batches
   bound to different device buffers, driven on two streams, overlap one
   batch's copies with the other's kernels as well. SLIC_ERR_STATE before
   slic_batch_set_buffers. */
slic_status slic_batch_segment_host(slic_batch b, const uint8_t *const *host_images, int32_t *const *host_labels,
                                    float *const *host_centres, void *stream);

/* Launch shape of the persistent assignment kernels: resident CTAs per SM
   (0 = as many as fit, capped by each kernel's occupancy), the number of
   TMA pipeline stages (3 or 4; 0 keeps the current value, default 4 where it
   fits), the row groups per warp (1: 256 threads, 4 pixels per thread;
   2: 128 threads per 32 tile rows, 8 pixels per thread, only when every
   frame's S is a multiple of 8; 0 keeps the current value, default 1) and
   the tile shape (tile_h = 32: 32x32-pixel tiles; 64: 32x64-pixel tiles,
   256 threads, two row groups only; 0 keeps the current value, default 32).
   SLIC_ERR_INVALID for other values or shapes that do not fit in shared
   memory. */
slic_status slic_batch_set_tuning(slic_batch b, int ctas_per_sm, int stages, int rows, int tile_h);

/* Fused passes (enable = 1; the default is 0, the autotuner chooses): with
   the pipelined kernel, the
   assignment passes before the last and the centre updates after them
   (Sec. 3 "Updating the cluster center", Sec. 4's loop) run as one
   cooperative launch. In every pass each CTA takes a contiguous block of
   the batch's tiles (frame after frame) and then the same share of the
   frames' update work (chunks of 256 centres), so the CTAs that sum a
   frame's pixels also update its centres. A frame's update starts when its
   tiles of the pass are summed, and its tiles of the next pass start when
   its update is done (per-frame phase counters; every wait is bounded, and
   one that gives up is reported by slic_batch_status as SLIC_ERR_TIMEOUT).
   No device-wide step separates the passes: one frame can be a pass ahead
   of another. enable = 0: one launch per pass and per update. Results are
   bit-identical either way. SLIC_ERR_INVALID for enable not 0 or 1. */
slic_status slic_batch_set_fused(slic_batch b, int enable);

/* Frame groups (1 .. min(4, n_frames); default 1): the batch runs as
   `groups` runs of consecutive frames of about equal pixel count, each
   enqueued on its own stream (the caller's stream for the first, streams of
   the batch for the others, forked from the caller's stream and joined back
   to it by events, so the call stays stream-ordered and can be captured in
   a CUDA graph). The groups' kernels run concurrently, so one group's pass
   boundaries (the last tiles of a pass, the update) overlap another group's
   passes. Results are bit-identical for any grouping. The learned warm
   start, component connectivity (mode 2), the non-pipelined kernels and
   profiling (slic_batch_profile_enable) run the batch as one group, as do
   fused passes. A change after the buffers are bound waits for the device.
   SLIC_ERR_INVALID outside the range. */
slic_status slic_batch_set_groups(slic_batch b, int groups);

/* Autotuner: time slic_batch_segment on the bound buffers for every launch
   shape that fits (3 timed runs each, CUDA events on `stream`; this waits
   for the device), keep the fastest, and append it to the JSON-lines file
   cache_path (may be NULL) under a key of GPU name, frame count,
   iterations and the distinct (width, height, S). When the key is already
   in the file its entry is used without timing. The search covers tile
   shapes x row groups per warp x pipeline stages x CTAs per SM x fused
   passes or not (slic_batch_set_fused) x frame groups (1, 2 or 4;
   slic_batch_set_groups); the choice is set on the batch and returned in
   *ctas_per_sm, *stages, *rows, *tile_h, *fused and *groups (any may be
   NULL). */
slic_status slic_batch_autotune(slic_batch b, const char *cache_path, void *stream, int *ctas_per_sm, int *stages,
                               int *rows, int *tile_h, int *fused, int *groups);

/* Pixels of all frames, kernel launches enqueued so far, and the launch
   shape of the assignment passes: CTAs per SM (as requested, capped by what
   fits), pipeline stages, row groups per warp, tile rows, fused passes and
   frame groups (stages and rows 0, tile rows 32, fused 0 when the
   pipelined kernel is not used); any pointer may be NULL. */
slic_status slic_batch_info(slic_batch b, long long *total_pixels, long long *launches, int *ctas_per_sm,
                            int *stages, int *rows, int *tile_h, int *fused, int *groups);

/* Grid of frame `frame` (Sec. 2): its S and ns_c x ns_r cells, K_eff =
   ns_c*ns_r centres (any pointer may be NULL); SLIC_ERR_INVALID for a frame
   index outside [0, n_frames). */
slic_status slic_batch_grid(slic_batch b, int frame, int *S, int *ns_c, int *ns_r);

/* Wait for the device, then report whether a bounded wait inside the
   batch's kernels gave up since the last call (SLIC_ERR_TIMEOUT; the
   affected tiles' results are then incomplete). Clears the flag. */
slic_status slic_batch_status(slic_batch b);

/* Wait for the device, then write each frame's number of centre updates in
   the last slic_batch_segment call to out[0 .. n_frames-1] (the stopping
   test is per frame: a frame that passed it skips its tiles in the
   remaining middle passes while the others go on). */
slic_status slic_batch_iterations_run(slic_batch b, int *out);

/* Device time of the batch's assignment launches, as slic_profile_enable /
   slic_profile_read do for a handle. */
slic_status slic_batch_profile_enable(slic_batch b, int enable);
slic_status slic_batch_profile_read(slic_batch b, double *assign_ms, long long *assign_launches);
/* The same records one by one, in enqueue order, for each
   slic_batch_segment call: with fused passes (slic_batch_set_fused) the
   fused launch (passes 0 .. iterations-1 and their updates) and the last
   pass, otherwise pass 0, 1, ..., iterations. Up to max_n durations (ms)
   into ms[], their number into *n. */
slic_status slic_batch_profile_times(slic_batch b, double *ms, int max_n, int *n);

/* Release the batch (waits for the device first). NULL is accepted. */
slic_status slic_batch_destroy(slic_batch b);

/* Reason for the last failure of this batch (or of the last failed
   slic_batch_create on this thread when b is NULL). Never NULL. */
const char *slic_batch_last_error(slic_batch b);

/* Allocation-free variant of slic_segment. The paper has no counterpart:
   it exists for callers that cannot allocate device memory (code running
   while a stream is captured into a CUDA graph, processes whose device
   memory belongs to another allocator with a fixed budget, loops that
   cannot afford the device synchronisation of cudaMalloc/cudaFree). It
   takes the parameters directly (no handle) and the same image, label and
   centre buffers, calls no cudaMalloc/cudaFree, and keeps its scratch in a
   32 MiB array in device memory that each GPU loading this library holds
   until the process exits. Images whose scratch exceeds 32 MiB are rejected
   with SLIC_ERR_INVALID; the scratch is 256 + 12*height*P + 48*K_eff +
   4*width*height bytes (P = width rounded up to 4), plus
   16*width*height + 8*ceil(width*height/32) + 4*ceil(width*height/65536) +
   256 with enforce_connectivity = 2, each part rounded up to 256 (plus a 256-byte
   state record). That
   admits e.g. 1280x720 or 1024x1024 at S >= 4 with connectivity mode 0 or
   1, and 1280x720 in mode 2; 1024x1024 in mode 2 and 1920x1080 in any mode
   do not fit. The first call on each device does a one-time set-up (sRGB
   table upload, kernel attributes) and should come before any stream
   capture. All calls share the one array: calls whose work overlaps on the
   GPU (different streams, or several host threads) race and corrupt each
   other's results; serialise them. The sums left by the previous call are
   cleared by each call. Errors are reported through slic_last_error(NULL);
   a bounded loop of component connectivity that gives up is reported by
   slic_noalloc_status_check. */
slic_status slic_segment_noalloc(const slic_params *params, const uint8_t *d_image, int32_t *d_labels,
                                 float *d_centres, void *stream);

/* Wait for the current device, then report whether a bounded loop of the
   allocation-free path's component connectivity (enforce_connectivity = 2)
   gave up since the last check on this device (SLIC_ERR_TIMEOUT: those
   labels are incomplete). Clears the flag. */
slic_status slic_noalloc_status_check(void);

/* ---- Fault injection, for tests of failure detection ----------------------
   (The paper has none.) Process-wide switches that make the library's own
   failure paths run without faulting the GPU:
     SLIC_FAULT_ALLOC         the value-th device allocation the library
                              makes from now on fails (that call frees what
                              it allocated before and returns
                              SLIC_ERR_NOMEM); 0 clears.
     SLIC_FAULT_WALK_LIMIT    component connectivity's bounded walks give up
                              after `value` steps instead of 2^22 (0 restores
                              it): deeper trees then report SLIC_ERR_TIMEOUT
                              through slic_status_check, slic_batch_status or
                              slic_noalloc_status_check.
     SLIC_FAULT_ABORT_COPIES  value != 0: the pipelined assignment kernel's
                              producers issue no further tile copy (checked
                              before each copy, so none is in flight when a
                              CTA gives up); the consumers' bounded waits run
                              out after about a second per launch and
                              slic_batch_status reports SLIC_ERR_TIMEOUT.
                              0 clears.
   The device words apply to the current device. SLIC_ERR_INVALID for an
   unknown kind or a negative value. */
typedef enum {
    SLIC_FAULT_ALLOC = 1,
    SLIC_FAULT_WALK_LIMIT = 2,
    SLIC_FAULT_ABORT_COPIES = 3
} slic_fault;
slic_status slic_fault_inject(int kind, long long value);

/* ---- Learned warm start ---------------------------------------------------
   A 4-layer 3x3 convolutional network (14 -> 32 -> 32 -> 32 -> 9 channels,
   ReLU between layers, zero padding; bfloat16 weights and stored
   activations, FP32 accumulation on the tensor cores) that predicts, for
   each pixel of an RGB image, logits over the 9 cells of its 3x3 cell
   window (slot t = (dy+1)*3 + (dx+1), the scan order of the assignment).
   Inputs per pixel (14): L/100, a/128, b/128, (x mod S)/S, (y mod S)/S and,
   for each slot, D/100 = the Eq. (1) distance to that cell's
   grid-initialised centre (2.0 off the grid). The
   paper has no such network; it replaces the first k-means iterations
   (its labels give initial centres through slic_update). Trained here by
   softmax cross-entropy against the slots of reference labels, with Adam
   (beta 0.9/0.999, eps 1e-8) on FP32 master weights. */
typedef struct slic_net_ctx *slic_net;

/* Network for batches of up to max_batch RGB images of width x height, grid
   interval S and compactness m (used by the distance inputs); He-normal
   weights from `seed`, zero biases. Allocates the activations of max_batch
   images. */
slic_status slic_net_create(int max_batch, int width, int height, int S, float m, unsigned long long seed,
                            slic_net *out);
slic_status slic_net_destroy(slic_net n);

/* Number of parameters (real sizes): per layer W[3][3][Cin][Cout] then b[Cout]. */
slic_status slic_net_param_count(slic_net n, size_t *count);

/* Host copies of the FP32 master weights (which = 0) or of the gradients of
   the last slic_net_gradients/slic_net_train_step (which = 1), in the order
   of slic_net_param_count; `count` must equal it. Synchronous. */
slic_status slic_net_get_params(slic_net n, int which, float *h_out, size_t count);
/* Load master weights (e.g. a checkpoint); synchronous. */
slic_status slic_net_set_params(slic_net n, const float *h_in, size_t count);

/* Inference on `batch` images d_images uint8 [batch][H][W][3]: d_logits
   float [batch][H][W][16] (first 9 used; may be NULL), d_labels int32
   [batch][H][W] = the label of the highest-scoring in-grid slot (may be
   NULL). */
slic_status slic_net_forward(slic_net n, int batch, const uint8_t *d_images, float *d_logits, int32_t *d_labels,
                             void *stream);

/* Forward and backward for targets d_targets uint8 [batch][H][W] (slots
   0..8, in-grid): gradients of the mean cross-entropy are kept for
   slic_net_get_params(which = 1); d_stats (may be NULL) receives float [2] =
   (sum of per-pixel losses, number of pixels whose argmax equals the
   target). */
slic_status slic_net_gradients(slic_net n, int batch, const uint8_t *d_images, const uint8_t *d_targets,
                               float *d_stats, void *stream);

/* slic_net_gradients, then one Adam step with learning rate lr. */
slic_status slic_net_train_step(slic_net n, int batch, const uint8_t *d_images, const uint8_t *d_targets, float lr,
                                float *d_stats, void *stream);

/* Training targets from labels: d_labels int32 [batch][H][W] (labels of
   the network's geometry, e.g. full-iteration SLIC labels before
   connectivity) -> d_slots uint8 [batch][H][W], the slot (dy+1)*3 + (dx+1)
   of each label's cell relative to the pixel's own cell. A label outside the
   pixel's 3x3 cell window gets slot 255 and adds 1 to *d_bad (a device int
   the caller clears; may be NULL). Enqueued on `stream`. */
slic_status slic_net_slots(slic_net n, int batch, const int32_t *d_labels, uint8_t *d_slots, int *d_bad,
                           void *stream);

/* Learned warm start of a segmentation (the paper has none; it replaces the
   first k-means iterations). Once armed with a network (NULL disarms), each
   slic_segment / slic_batch_segment call runs, after the colour conversion
   and the initialisation: the network's labels for the frame, then one
   update from them (Sec. 3 "Updating the cluster center": each centre
   becomes the mean of the pixels the network gave its cell; a cell given no
   pixel keeps its initial centre, from the grid or from
   slic_set_init_centres / d_init), then the usual passes: assignment,
   `iterations` x {update, assignment}, connectivity. The network must have
   been created for the frames' width, height, S and m (else
   SLIC_ERR_INVALID); it is read by every later call and must outlive the
   arming. Its forward runs in chunks of its max_batch images; frames may
   have 3 or 4 channels (all frames of a batch the same). The batch form
   waits for the device and allocates the network's label maps (4 bytes per
   pixel) the first time it is armed; the per-frame results equal those of
   the armed single-frame handle bit for bit. */
slic_status slic_set_warmstart(slic_handle h, slic_net net);
slic_status slic_batch_set_warmstart(slic_batch b, slic_net net);

/* Wait for the device, then report whether a bounded wait inside the
   network's tensor-core kernels gave up since the last call
   (SLIC_ERR_TIMEOUT; that forward pass's outputs are then incomplete).
   Clears the flag. */
slic_status slic_net_status(slic_net n);

const char *slic_net_last_error(slic_net n);

/* Reason for the last failure on this handle (or of the last failed
   slic_create on this thread when h is NULL). Never NULL. */
const char *slic_last_error(slic_handle h);

#ifdef __cplusplus
}
#endif

#endif /* SLIC_H */
