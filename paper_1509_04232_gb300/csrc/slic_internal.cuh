// Internal declarations shared by the kernels and the C-ABI layer of
// libslicgb.so. Not part of the public interface (that is include/slic.h).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "slic.h"

namespace slicgb {

// Fixed-point scale for the centre-update sums: CIELAB and XYZ features
// (|f| < 128) are rounded to multiples of 2^-15 before summation, RGB
// features are integers already (scale 1). Every partial sum is then an
// exact integer, so the result does not depend on summation order, tiling
// or batching. |f| * 2^15 < 2^22 lets the pipelined kernel round on the FMA
// pipe (fix_round2); a centre moves by at most 2^-16 from the exact mean.
constexpr float kFixScaleFrac = 32768.0f;

// Assignment tile: 32 x 32 pixels, 256 threads, 4 horizontally adjacent
// pixels per thread.
constexpr int kTileW = 32;
constexpr int kTileH = 32;
constexpr int kPPT = 4;
constexpr int kThreads = (kTileW / kPPT) * kTileH;

// Record of the padded centre table read by the pipelined assignment: every
// field twice, (L, L, a, a, b, b, x, x, y, y, n, 0), so that the paired
// (two pixels per instruction) FP32 arithmetic takes a centre field as one
// 64-bit operand.
constexpr int kCtabRec = 12;

// Colour-conversion constants, computed on the host in double precision and
// rounded to float (see slic_api.cu).
struct ConvConsts {
    float m[9];       // linear sRGB -> (X/Xn, Y/Yn, Z/Zn) for CIELAB, or XYZ*100
    float eps;        // CIE epsilon 216/24389
    float k_slope;    // kappa/116
    float k_offset;   // 16/116
    int color_space;  // 0 CIELAB, 1 RGB, 2 XYZ
};

#ifdef __CUDACC__
// Cube root of t > 0 from the identity t^(1/3) = 2^(log2(t) / 3), with the
// hardware base-2 logarithm and exponential approximations (relative error
// a few 1e-7 over CIELAB's range t in (216/24389, 1.1]).
static __device__ __forceinline__ float cbrt_exp2(float t) {
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(t));
    l *= (1.0f / 3.0f);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(l));
    return r;
}

static __device__ __forceinline__ float lab_f(const ConvConsts &cc, float t) {
    return t > cc.eps ? cbrt_exp2(t) : fmaf(cc.k_slope, t, cc.k_offset);
}

// Sec. 3 "Image space conversion" for one pixel. `lut` is the sRGB
// linearisation table (shared or global memory).
static __device__ __forceinline__ void convert_pixel(const ConvConsts &cc, unsigned r, unsigned g, unsigned b,
                                              const float *lut, float &f0, float &f1, float &f2) {
    if (cc.color_space == 1) {
        f0 = (float)r;
        f1 = (float)g;
        f2 = (float)b;
        return;
    }
    const float lr = lut[r], lg = lut[g], lb = lut[b];
    const float *m = cc.m;
    const float X = fmaf(m[0], lr, fmaf(m[1], lg, m[2] * lb));
    const float Y = fmaf(m[3], lr, fmaf(m[4], lg, m[5] * lb));
    const float Z = fmaf(m[6], lr, fmaf(m[7], lg, m[8] * lb));
    if (cc.color_space == 2) {
        f0 = X;
        f1 = Y;
        f2 = Z;
        return;
    }
    const float fx = lab_f(cc, X), fy = lab_f(cc, Y), fz = lab_f(cc, Z);
    f0 = fmaf(116.0f, fy, -16.0f);
    f1 = 500.0f * (fx - fy);
    f2 = 200.0f * (fy - fz);
}

#endif

// Per-frame state of the stopping test (Sec. 2: the iteration ends once
// the centres stabilise, read as the mean L1 move of their positions): the
// sums of |dx| + |dy| over the centres in fixed point (scale kResidScale,
// so the sums are exact whatever the order) for three consecutive updates
// (slot = update index mod 3), each spread over kResidLanes counters so
// that a frame's warps do not all add to one address, the stop flag and the
// updates performed.
constexpr int kResidLanes = 8;
struct ConvState {
    long long resid[3][kResidLanes];
    int done;
    int iters;
    // Phase counters of the fused multi-pass assignment (reset with the
    // rest by the initialisation): tiles of this frame whose sums are in the
    // global sums, and warps that finished their part of an update chunk,
    // both counted over all passes of one launch.
    int tiles_done;
    int chunks_done;
};
constexpr float kResidScale = 65536.0f;

// One frame's geometry and buffers as seen by the kernels (a kernel
// parameter for single-frame launches, an entry of a device-side table for
// batched ones).
struct FrameArgs {
    CUtensorMap feat_map;   // features as a [3][H][P] f32 tensor, box 32x32x3 (batched path)
    CUtensorMap ctab_map;   // padded centre table as [(ns_r+2)][(ns_c+2)*kCtabRec] f32, box box_w*kCtabRec x box_h
    CUtensorMap feat_map64; // the same for 32x64 tiles: box 32x64x3, and
    CUtensorMap ctab_map64; // box box_w*kCtabRec x box_h64
    ConvConsts conv;
    const uint8_t *rgb;     // [H][W][C]
    float *feat;            // 3 planes [H][P]; plane stride H*P
    const float *centres;   // [K][6] read by the assignment
    float *centres_out;     // [K][6] written by init and update
    long long *acc;         // [K][6] fixed-point sums (l,a,b scaled; x,y,count exact)
    int32_t *labels;        // [H][W]
    int32_t *lbl_tmp;       // [H][W] connectivity ping-pong (batched path)
    const float *init;      // [K][6] initial centres instead of the grid (batched path)
    float *ctab;            // [(ns_r+2)(ns_c+2)][kCtabRec] centres with a sentinel ring (batched path)
    int W, H, P, C, S, ns_c, ns_r;
    float w;                // m / S
    int win_max;            // largest centre window of any tile (sizes shared memory)
    int direct_acc;         // 1: partial sums go straight to global atomics
    int rgb_vec;            // 1: image rows allow 4-pixel vector loads
    int labels_vec;         // 1: label rows allow 4-pixel vector stores
    float fix_scale;        // fixed-point scale of the feature sums
    unsigned s_mul;         // ceil(2^32 / S) for S <= 2048, else 0
    int tiles_x;            // 32x32 tiles per row
    int tile_base;          // first tile / centre / row of this frame in the
    int centre_base;        // batch's concatenated lists (0 for a single
    int row_base;           // frame)
    int box_w, box_h;       // window box of the centre-table copies (cells)
    int tile_base64, box_h64;  // the frame's first 32x64 tile; window rows of a 32x64 tile
    int32_t *assign_out;    // labels of the pipelined last pass (lbl_tmp when the
    int assign_vec;         // fused connectivity follows); 1: 4-pixel vector stores
    int strips_x;           // fused connectivity: strips per row and first
    int strip_base;         // work unit (strip x row segment) of this frame
    int perturb;            // 1: grid seeds move to the lowest-gradient pixel nearby (Sec. 2)
    float conv_eps;         // stopping threshold on the mean L1 move (0: fixed iterations)
    ConvState *cstate;      // the frame's stopping-test state (reset by the initialisation)
    const int32_t *init_labels;  // [H][W] labels whose member means replace the grid
                                 // centres (learned warm start), or null
    // Fused multi-pass assignment: the frame's tiles per tile height, its
    // update chunks (kUpdateChunk centres each) and its first chunk in the
    // batch's list of chunks
    int n_tiles, n_tiles64, n_chunks;
    int chunk_base;
};
constexpr int kUpdateChunk = 256;  // centres per update work item of the fused assignment

// Shared memory for one assignment CTA whose tile spans at most win_n cells.
size_t assign_smem_bytes(int win_n, bool first);
int assign_max_window(int S, int ns_c, int ns_r, int tile_h = 32);
bool assign_direct_acc(int win_n);
// Resident CTAs per SM of the batched assignment kernel.
int assign_batch_occupancy(bool same, size_t smem);

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point
// query, once); nullptr if the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Host helpers shared by the C-ABI files: colour constants of a feature
// space, and the once-per-device set-up (sRGB table, shared-memory limit).
ConvConsts conv_consts(int color_space);
void srgb_table(float lut[256]);
cudaError_t device_setup(int dev, size_t smem);

cudaError_t upload_lut(const float *lut256);

// Device allocations of the library go through dev_malloc, so that fault
// injection (slic_fault_inject, SLIC_FAULT_ALLOC) can make them fail.
cudaError_t dev_malloc(void **p, size_t bytes);
template <typename T>
cudaError_t dev_alloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
// The device words of fault injection on the current device: the step limit
// of component connectivity's walks and the pipelined assignment's copy stop.
cudaError_t set_fault_words(unsigned ccl_steps, int abort_copies);
unsigned ccl_default_steps();
cudaError_t configure_kernels(size_t max_smem);

cudaError_t launch_init_from_rgb(const FrameArgs &a, cudaStream_t s);
cudaError_t launch_init_batch(const FrameArgs *d_frames, int n, int total_centres, cudaStream_t s);
cudaError_t launch_init_from_feat(const float *feat, int W, int H, int P, int S, int ns_c, int ns_r, int perturb,
                                  float *centres, cudaStream_t s);
cudaError_t launch_zero_acc(long long *acc, int K, cudaStream_t s);
// first: convert from RGB (and store features unless last); last: write labels
// instead of accumulating.
cudaError_t launch_assign(const FrameArgs &a, bool first, bool last, bool store_feat, size_t smem,
                          cudaStream_t s);
cudaError_t launch_assign_batch(const FrameArgs *d_frames, int n, int total_tiles, int win_max, bool same, bool first,
                                bool last, size_t smem, int grid, cudaStream_t s);
// Update `it` (1-based) of a run; with cstate (and eps > 0) it applies the
// stopping test first and records its move (cstate may be null: a plain
// update, as the stage-by-stage API does).
cudaError_t launch_update(long long *acc, const float *centres_in, float *centres_out, int K, float fix_inv,
                          ConvState *cstate, float eps, int it, cudaStream_t s);
cudaError_t launch_update_batch(const FrameArgs *d_frames, int n, int total_centres, int it, cudaStream_t s);
// Pipelined (TMA bulk copies, mbarrier) assignment for the passes after the
// first, reading features and the padded centre table; *err is set on a
// timed-out wait.
// rows = 1: 256 threads, 4 pixels per thread (ctas_per_sm >= 4 selects the
// 64-register build); rows = 2: 128 threads, 8 pixels per thread (two row
// groups in one cell row: every frame's S a multiple of 8, `same` set).
// check_stop: some frame has a stopping threshold (its tiles are then skipped
// once it has stopped). tile_h = 64 (rows = 2 only): 32x64 tiles, 256
// threads (8 warps of two row groups); total_tiles and win_max are then
// those of 32x64 tiles.
cudaError_t launch_assign_pipe(const FrameArgs *d_frames, int n, int total_tiles, int win_max, bool same, bool last,
                               int nst, int rows, int tile_h, int ctas_per_sm, int grid, int *err, int check_stop,
                               cudaStream_t s);
// Fused multi-pass form of the same kernel, one cooperative launch: passes
// 0 .. passes-1 with the update after each (updates 1 .. passes), ordered
// per frame by the phase counters in its ConvState (reset by the
// initialisation); the last pass is a separate launch_assign_pipe. Each CTA
// takes, in every pass, a contiguous block of the batch's total_tiles tiles
// (of tile_h rows) and the same share of its total_chunks update chunks.
// grid must not exceed the resident CTAs (a cooperative launch fails then).
cudaError_t launch_assign_multi(const FrameArgs *d_frames, int n, int total_tiles, int total_chunks, int win_max,
                                bool same, int passes, int nst, int rows, int tile_h, int ctas_per_sm, int grid,
                                int *err, int check_stop, cudaStream_t s);
// Shared memory and resident CTAs per SM of the pipelined kernel with nst
// (3..4) stages, 1 or 2 row groups per warp and tiles of tile_h rows (multi:
// the fused multi-pass build).
size_t assign_pipe_smem_bytes(int win_n, bool last, int nst, int rows, int tile_h = 32, bool multi = false);
int assign_pipe_occupancy(bool same, int win_n, int nst, int rows, int tile_h = 32, bool multi = false);
// Batched RGB -> features pre-pass (the pipelined path's first pass reads
// the features it writes).
cudaError_t launch_convert_batch(const FrameArgs *d_frames, int n, int total_rows, int max_w, cudaStream_t s);
cudaError_t launch_fill_ring(const FrameArgs *d_frames, int n, int max_ring, cudaStream_t s);
cudaError_t launch_accumulate_labels(const float *feat, int W, int H, int P, const int32_t *labels, int K,
                                     long long *acc, float fix_scale, cudaStream_t s);
// Member sums of every frame's init_labels map (frames without one are
// skipped); the sums must be zero before (the initialisation clears them).
cudaError_t launch_accumulate_labels_batch(const FrameArgs *d_frames, int n, int total_rows, int max_w,
                                           cudaStream_t s);
cudaError_t launch_convert(const ConvConsts &cc, const uint8_t *rgb, int W, int H, int C, float *feat, int P,
                           cudaStream_t s);
cudaError_t launch_connectivity(const int32_t *in, int32_t *out, int W, int H, cudaStream_t s);
cudaError_t launch_connectivity_batch(const FrameArgs *d_frames, int n, int total_rows, int max_w, int pass,
                                      cudaStream_t s);
// Both connectivity passes in one launch (a warp streams down a 120-column
// strip of a row segment): reads lbl_tmp, writes labels. Units of a frame
// (strips x segments) and its strips per row:
int connectivity2_units(int W, int H, int *strips_x);
cudaError_t launch_connectivity2_batch(const FrameArgs *d_frames, int n, int total_units, int grid, cudaStream_t s);
// Component-based connectivity (connectivity mode 2): in -> out over a W x H
// label map (out may equal in), segments of at most min_size pixels joined
// to a neighbour. scratch holds ccl_scratch_ints(W*H) ints; a bounded walk
// that gives up sets bit 1 of *err.
size_t ccl_scratch_ints(long long N);
cudaError_t launch_connectivity_components(const int32_t *in, int32_t *out, int W, int H, int min_size,
                                           int *scratch, int *err, cudaStream_t s);
// Several frames at once: d_table[n] (device) describes each frame, base =
// its first index in the concatenation of all frames' pixels (G in total,
// below 2^31) and tile_base its first 32x32 tile in the concatenation of all
// frames' tiles (`tiles` in total, ccl_tiles per frame); scratch holds
// ccl_scratch_ints(G) ints. For n == 1, `one` is used and d_table may be
// null.
struct CclFrame {
    const int32_t *in;
    int32_t *out;
    int W;
    int min_size;
    int base;
    int H;
    int tile_base;  // first 32x32 tile of the frame in the call's list of tiles
};
// 32x32 tiles of a W x H frame (the unit of the component stages).
int ccl_tiles(int W, int H);
cudaError_t launch_connectivity_components(const CclFrame *d_table, const CclFrame &one, int n, int G, int tiles,
                                           int *scratch, int *err, cudaStream_t s);
// The learned warm start's network (slic_net.cu) as seen by the segmentation
// drivers: its geometry, and the labels of `batch` images (uint8 [H][W][C],
// C = 3 or 4; given by a device table of image pointers, or contiguous in
// d_images when d_table is null) into labels [batch][H][W], forward passes
// of at most max_batch images (on failure slic_net_last_error tells why).
bool net_geometry(const slic_net_ctx *n, int *W, int *H, int *S, float *m, int *max_batch);
cudaError_t net_forward_labels(slic_net_ctx *n, int batch, const uint8_t *d_images, const uint8_t *const *d_table,
                               int C, int32_t *labels, cudaStream_t s);
// Event record for the profiling timers, valid inside and outside stream capture.
cudaError_t record_profile_event(cudaEvent_t ev, cudaStream_t s);

}  // namespace slicgb
