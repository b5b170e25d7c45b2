// SLIC kernels for sm_103a (gSLICr, arXiv 1509.04232, Sec. 3).
//
//   init      "Cluster center initialisation": one thread per centre; position
//             = midpoint of the in-image part of its grid cell, colour = the
//             pixel under it (converted on the fly).
//   assign    "Finding the cluster associations" (Eq. 1) for one 32x32-pixel
//             tile, with the tile's window of centres staged in shared memory.
//             The first pass fuses "Image space conversion" (RGB bytes in,
//             features stored once); every pass but the last fuses the first
//             half of "Updating the cluster center" (per-tile member sums,
//             flushed with one global atomic per centre component per tile).
//   update    second half of the update: centre = sums / count; an empty
//             centre keeps its position and colour.
//   connect   one pass of "Enforce connectivity".
//
// Every stage exists as a single-frame kernel (a frame's arguments are a
// __grid_constant__ parameter) and as a batched kernel over a table of frame
// descriptors in device memory (the assignment one persistent: a grid sized
// to the GPU loops over the tiles of all frames). The member sums are exact
// integers (features in fixed point), so results do not depend on the order
// in which tiles, warps or frames contribute: a frame segmented alone or in
// any batch gives bit-identical labels and centres.
#include "slic_internal.cuh"

#include <cstdint>

namespace slicgb {

__device__ float g_lut[256];  // sRGB byte -> linear, filled by the host

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarps = kThreads / 32;
constexpr float kSentinel = 1e18f;
constexpr size_t kPrivateAccLimit = 64 * 1024;

// One record of the padded centre table: each field twice (see kCtabRec).
__device__ __forceinline__ void write_ctab(float *t, const float *c) {
    float4 *t4 = reinterpret_cast<float4 *>(t);
    t4[0] = make_float4(c[0], c[0], c[1], c[1]);
    t4[1] = make_float4(c[2], c[2], c[3], c[3]);
    t4[2] = make_float4(c[4], c[4], c[5], 0.0f);
}

// Candidate tags 0..8 (scan position in the 3x3 window) for the keys
// (D & ~15) | t, read from the constant bank: the key is then one logical
// operation whose other constant, the mask, is its immediate. With the tag
// as a literal too, the pipelined pass executed 7 more instructions per
// pixel (ncu instruction counts; same results).
__constant__ unsigned c_tags[9] = {0, 1, 2, 3, 4, 5, 6, 7, 8};

__device__ __forceinline__ float fsqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// x / S for 0 <= x < 2^21 using the frame's multiplier ceil(2^32 / S) (exact
// for S <= 2048; s_mul == 0 selects a plain division).
__device__ __forceinline__ int div_s(int x, unsigned s_mul, int S) {
    return s_mul ? (int)__umulhi((unsigned)x, s_mul) : x / S;
}

// Index of the frame whose [base, next base) range holds `idx` (frames are
// sorted by base; base of frame 0 is 0).
enum BaseField { kTileBase, kCentreBase, kRowBase, kStripBase, kTileBase64, kChunkBase };
template <BaseField F>
__device__ __forceinline__ int base_of(const FrameArgs &a) {
    return F == kTileBase ? a.tile_base
           : F == kCentreBase ? a.centre_base
           : F == kRowBase ? a.row_base
           : F == kStripBase ? a.strip_base
           : F == kTileBase64 ? a.tile_base64
                              : a.chunk_base;
}
template <BaseField F>
__device__ __forceinline__ int find_frame(const FrameArgs *frames, int n, int idx) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base_of<F>(frames[mid]) <= idx)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Dynamic shared memory of an assignment CTA: window centres, per-warp
// private accumulators (unless the window is too large), sRGB table (first
// pass). Also the offset of the table when `first` is false.
__host__ __device__ __forceinline__ size_t smem_layout(int win_n, bool first) {
    size_t b = ((size_t)win_n * 20 + 15) & ~(size_t)15;
    if ((size_t)kWarps * win_n * 4 * sizeof(int) <= kPrivateAccLimit) b += (size_t)kWarps * win_n * 4 * sizeof(int);
    if (first) b += 256 * sizeof(float);
    return b;
}

}  // namespace

// ---------------------------------------------------------------------------
// Initialisation
// ---------------------------------------------------------------------------

__device__ __forceinline__ void init_centre_position(int k, int W, int H, int S, int ns_c, float &xk, float &yk,
                                                     int &px, int &py) {
    const int c = k % ns_c, r = k / ns_c;
    const int x_first = c * S, x_last = min((c + 1) * S, W) - 1;
    const int y_first = r * S, y_last = min((r + 1) * S, H) - 1;
    // (first + last) / 2 is exact in float for any image below 2^23 pixels wide.
    xk = 0.5f * (float)(x_first + x_last);
    yk = 0.5f * (float)(y_first + y_last);
    px = (x_first + x_last) >> 1;  // floor of the midpoint
    py = (y_first + y_last) >> 1;
}

// Seed perturbation (Sec. 2, the original SLIC's first step): the pixel of
// lowest gradient G = |I(x+1,y) - I(x-1,y)|^2 + |I(x,y+1) - I(x,y-1)|^2
// (features, neighbours clamped into the image) among the 3x3 pixels around
// the seed pixel (px, py). The seed pixel is the first candidate; a later
// one (dy outer, dx inner, in-image only) wins only with a strictly lower G.
// fetch(x, y, f) gives the features of an in-image pixel. Returns whether the
// seed moved, with the chosen pixel and its features.
template <typename Fetch>
__device__ __forceinline__ bool perturb_seed(const Fetch &fetch, int W, int H, int px, int py, int &bx, int &by,
                                             float (&fb)[3]) {
    float f[5][5][3];  // features of the 5x5 block around (px, py), clamped; corners unused
#pragma unroll
    for (int j = 0; j < 5; ++j) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if ((i == 0 || i == 4) && (j == 0 || j == 4)) continue;
            fetch(min(max(px - 2 + i, 0), W - 1), min(max(py - 2 + j, 0), H - 1), f[j][i]);
        }
    }
    auto grad = [&](int i, int j) {
        float g = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float gx = f[j][i + 1][c] - f[j][i - 1][c], gy = f[j + 1][i][c] - f[j - 1][i][c];
            g += gx * gx + gy * gy;
        }
        return g;
    };
    float best = grad(2, 2);
    int bi = 2, bj = 2;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            if ((dx == 0 && dy == 0) || px + dx < 0 || px + dx >= W || py + dy < 0 || py + dy >= H) continue;
            const float g = grad(2 + dx, 2 + dy);
            if (g < best) {
                best = g;
                bi = 2 + dx;
                bj = 2 + dy;
            }
        }
    }
    bx = px + bi - 2;
    by = py + bj - 2;
#pragma unroll
    for (int c = 0; c < 3; ++c) fb[c] = f[bj][bi][c];
    return bi != 2 || bj != 2;
}

__device__ __forceinline__ void init_centre(const FrameArgs &a, int k) {
    float xk, yk;
    int px, py;
    init_centre_position(k, a.W, a.H, a.S, a.ns_c, xk, yk, px, py);
    float fv[3];
    if (a.perturb) {
        int bx, by;
        auto fetch = [&](int x, int y, float (&o)[3]) {
            const uint8_t *q = a.rgb + ((size_t)y * a.W + x) * a.C;
            convert_pixel(a.conv, q[0], q[1], q[2], g_lut, o[0], o[1], o[2]);
        };
        if (perturb_seed(fetch, a.W, a.H, px, py, bx, by, fv)) {
            xk = (float)bx;
            yk = (float)by;
        }
    } else {
        const uint8_t *p = a.rgb + ((size_t)py * a.W + px) * a.C;
        convert_pixel(a.conv, p[0], p[1], p[2], g_lut, fv[0], fv[1], fv[2]);
    }
    float *ck = a.centres_out + (size_t)k * 6;
    ck[0] = fv[0];
    ck[1] = fv[1];
    ck[2] = fv[2];
    ck[3] = xk;
    ck[4] = yk;
    ck[5] = 0.0f;
    long long *ak = a.acc + (size_t)k * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) ak[c] = 0;
}

__device__ __forceinline__ void reset_conv(ConvState *cs) {
    if (cs) {
#pragma unroll
        for (int i = 0; i < 3 * kResidLanes; ++i) (&cs->resid[0][0])[i] = 0;
        cs->done = 0;
        cs->iters = 0;
        cs->tiles_done = 0;
        cs->chunks_done = 0;
    }
}

__global__ void k_init_rgb(const __grid_constant__ FrameArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < a.ns_c * a.ns_r) init_centre(a, k);
    if (k == 0) reset_conv(a.cstate);
}

// Batched initialisation; a frame with `init` set copies those centres
// (e.g. the previous video frame's) instead of the grid initialisation.
__global__ void k_init_batch(const FrameArgs *frames, int n, int total) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    // one frame lookup per warp, a lane's own only across a frame boundary
    const int g0 = __shfl_sync(__activemask(), g, 0);
    int f = find_frame<kCentreBase>(frames, n, g0);
    if (f + 1 < n && g >= frames[f + 1].centre_base) f = find_frame<kCentreBase>(frames, n, g);
    const FrameArgs &a = frames[f];
    const int k = g - a.centre_base;
    if (a.init) {
#pragma unroll
        for (int c = 0; c < 6; ++c) a.centres_out[(size_t)k * 6 + c] = a.init[(size_t)k * 6 + c];
#pragma unroll
        for (int c = 0; c < 6; ++c) a.acc[(size_t)k * 6 + c] = 0;
    } else {
        init_centre(a, k);
    }
    if (k == 0) reset_conv(a.cstate);
    if (a.ctab) {
        const int r = k / a.ns_c, c = k - (k / a.ns_c) * a.ns_c;
        write_ctab(a.ctab + ((size_t)(r + 1) * (a.ns_c + 2) + c + 1) * kCtabRec, a.centres_out + (size_t)k * 6);
    }
}

// Sentinel ring of the padded centre tables (ring index i of frame f).
__global__ void k_fill_ring(const FrameArgs *frames, int n, int max_ring) {
    const int f = blockIdx.y;
    if (f >= n) return;
    const FrameArgs &a = frames[f];
    const int cw = a.ns_c + 2, ch = a.ns_r + 2;
    const int ring = 2 * cw + 2 * (ch - 2);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ring && i < max_ring; i += gridDim.x * blockDim.x) {
        int r, c;
        if (i < cw) { r = 0; c = i; }
        else if (i < 2 * cw) { r = ch - 1; c = i - cw; }
        else { const int j = i - 2 * cw; r = 1 + (j >> 1); c = (j & 1) ? cw - 1 : 0; }
        float4 *t = reinterpret_cast<float4 *>(a.ctab + ((size_t)r * cw + c) * kCtabRec);
#pragma unroll
        for (int q = 0; q < kCtabRec / 4; ++q) t[q] = make_float4(1e18f, 1e18f, 1e18f, 1e18f);
    }
}

__global__ void k_init_feat(const float *feat, int W, int H, int P, int S, int ns_c, int ns_r, int perturb,
                            float *centres) {
    const int K = ns_c * ns_r;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    float xk, yk;
    int px, py;
    init_centre_position(k, W, H, S, ns_c, xk, yk, px, py);
    const size_t plane = (size_t)H * P;
    auto fetch = [&](int x, int y, float (&o)[3]) {
        const size_t off = (size_t)y * P + x;
        o[0] = feat[off];
        o[1] = feat[plane + off];
        o[2] = feat[2 * plane + off];
    };
    float fv[3];
    int bx, by;
    if (perturb && perturb_seed(fetch, W, H, px, py, bx, by, fv)) {
        xk = (float)bx;
        yk = (float)by;
    } else {
        fetch(px, py, fv);
    }
    float *ck = centres + (size_t)k * 6;
    ck[0] = fv[0];
    ck[1] = fv[1];
    ck[2] = fv[2];
    ck[3] = xk;
    ck[4] = yk;
    ck[5] = 0.0f;
}

__global__ void k_zero_acc(long long *acc, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] = 0;
}

// ---------------------------------------------------------------------------
// Assignment (+ fused conversion and partial update sums)
// ---------------------------------------------------------------------------
//
// A tile is 32x32 pixels handled by 8 warps; warp w covers the 16x8 block at
// (16*(w%2), 8*(w/2)) of the tile and lane l the 4 horizontally adjacent
// pixels at (4*(l%4), l/4) of that block, so a warp reads 8 rows of 64
// contiguous bytes per feature plane.

// Window of cells a tile can reference: the cells its pixels fall in plus
// one ring, clamped to what the grid can offer.
int assign_max_window(int S, int ns_c, int ns_r, int tile_h) {
    const int span = (kTileW - 1) / S + 2;  // cells a 32-px run can touch, misaligned
    const int spanh = (tile_h - 1) / S + 2;
    const int wx = (span < ns_c ? span : ns_c) + 2;
    const int wy = (spanh < ns_r ? spanh : ns_r) + 2;
    return wx * wy;
}

bool assign_direct_acc(int win_n) { return (size_t)kWarps * win_n * 4 * sizeof(int) > kPrivateAccLimit; }

size_t assign_smem_bytes(int win_n, bool first) { return smem_layout(win_n, first); }

namespace {

// Warp-aggregated accumulation of one value set per lane into the global
// sums, keyed by window index (key < 0: no contribution). All 32 lanes must
// call it. Used only when the window is too large for private accumulators.
__device__ __forceinline__ void warp_accumulate(int key, const int (&v)[6], unsigned long long *gacc, int wx0,
                                                int wy0, int wnx, int ns_c) {
    const int lane = threadIdx.x & 31;
    unsigned pending = __ballot_sync(kFull, key >= 0);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int k = __shfl_sync(kFull, key, leader);
        const bool mine = (key == k);
        const unsigned grp = __ballot_sync(kFull, mine);
        const int r0 = __reduce_add_sync(kFull, mine ? v[0] : 0);
        const int r1 = __reduce_add_sync(kFull, mine ? v[1] : 0);
        const int r2 = __reduce_add_sync(kFull, mine ? v[2] : 0);
        const int r3 = __reduce_add_sync(kFull, mine ? v[3] : 0);
        const int r4 = __reduce_add_sync(kFull, mine ? v[4] : 0);
        const int r5 = __reduce_add_sync(kFull, mine ? v[5] : 0);
        if (lane < 6) {
            const int val = lane == 0 ? r0 : lane == 1 ? r1 : lane == 2 ? r2 : lane == 3 ? r3 : lane == 4 ? r4 : r5;
            const int cell = (wy0 + k / wnx) * ns_c + (wx0 + k % wnx);
            atomicAdd(&gacc[(size_t)cell * 6 + lane], (unsigned long long)(long long)val);
        }
        pending &= ~grp;
    }
}

// Merge runs of equal keys among a lane's kPPT pixels, then reduce each run
// across the warp and add it to the global sums (all 32 lanes must call it).
__device__ __forceinline__ void accumulate_runs(const int (&key)[kPPT], int (&v)[kPPT][6], unsigned long long *gacc,
                                                int wx0, int wy0, int wnx, int ns_c) {
#pragma unroll
    for (int j = kPPT - 2; j >= 0; --j) {
        if (key[j + 1] == key[j]) {
#pragma unroll
            for (int c = 0; c < 6; ++c) v[j][c] += v[j + 1][c];
        }
    }
#pragma unroll
    for (int j = 0; j < kPPT; ++j) {
        const int k = (j == 0 || key[j] != key[j - 1]) ? key[j] : -1;
        if (__any_sync(kFull, k >= 0)) warp_accumulate(k, v[j], gacc, wx0, wy0, wnx, ns_c);
    }
}

}  // namespace

// One assignment pass over the tile at (tx0, ty0) of frame `fa`.
//   FIRST: features come from the RGB bytes (and are stored for later passes).
//   LAST:  labels are written; otherwise every centre's member sums are
//          accumulated for the update (exact integers).
//   SAME:  S is a multiple of kPPT, so a thread's kPPT pixels share a cell.
// `smem` is the CTA's dynamic shared memory; `lut` (FIRST) holds the sRGB
// table. The caller must __syncthreads() before reusing shared memory.
template <bool FIRST, bool LAST, bool SAME>
__device__ __forceinline__ void assign_tile(const FrameArgs &fa, int tx0, int ty0, int store_feat,
                                            unsigned char *smem, const float *lut) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = fa.W, H = fa.H, S = fa.S, P = fa.P, C = fa.C, ns_c = fa.ns_c, ns_r = fa.ns_r;
    const int win_max = fa.win_max;
    const unsigned s_mul = fa.s_mul;
    const bool direct = fa.direct_acc != 0;
    const float *const feat_in = fa.feat;
    float *const feat_out = fa.feat;

    // Window of centres for this tile.
    const int ccx0 = div_s(tx0, s_mul, S), ccx1 = div_s(min(tx0 + kTileW - 1, W - 1), s_mul, S);
    const int ccy0 = div_s(ty0, s_mul, S), ccy1 = div_s(min(ty0 + kTileH - 1, H - 1), s_mul, S);
    const int wx0 = ccx0 - 1, wy0 = ccy0 - 1;
    const int wnx = ccx1 - ccx0 + 3, wny = ccy1 - ccy0 + 3;
    const int nwin = wnx * wny;

    float4 *cA = reinterpret_cast<float4 *>(smem);
    float *cY = reinterpret_cast<float *>(cA + nwin);
    unsigned *wacc = reinterpret_cast<unsigned *>(smem + (((size_t)win_max * 20 + 15) & ~(size_t)15));

    // Pixels of this thread; their loads are issued before the staging
    // barrier so both latencies overlap.
    const int x = tx0 + 16 * (warp & 1) + 4 * (lane & 3);
    const int y = ty0 + 8 * (warp >> 1) + (lane >> 2);
    const bool row_ok = (y < H) && (x < W);
    const size_t plane = (size_t)H * P;
    const size_t foff = (size_t)y * P + x;
    float f0[kPPT] = {}, f1[kPPT] = {}, f2[kPPT] = {};
    unsigned rgbw[4] = {0u, 0u, 0u, 0u};
    if (row_ok) {
        if (FIRST) {
            if (fa.rgb_vec) {
                const uint8_t *p = fa.rgb + ((size_t)y * W + x) * C;
                if (C == 3) {
                    const uint32_t *q = reinterpret_cast<const uint32_t *>(p);
                    rgbw[0] = __ldg(q);
                    rgbw[1] = __ldg(q + 1);
                    rgbw[2] = __ldg(q + 2);
                } else {
                    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
                    rgbw[0] = q.x;
                    rgbw[1] = q.y;
                    rgbw[2] = q.z;
                    rgbw[3] = q.w;
                }
            }
        } else if ((P & 3) == 0) {
            const float4 v0 = __ldg(reinterpret_cast<const float4 *>(feat_in + foff));
            const float4 v1 = __ldg(reinterpret_cast<const float4 *>(feat_in + plane + foff));
            const float4 v2 = __ldg(reinterpret_cast<const float4 *>(feat_in + 2 * plane + foff));
            f0[0] = v0.x; f0[1] = v0.y; f0[2] = v0.z; f0[3] = v0.w;
            f1[0] = v1.x; f1[1] = v1.y; f1[2] = v1.z; f1[3] = v1.w;
            f2[0] = v2.x; f2[1] = v2.y; f2[2] = v2.z; f2[3] = v2.w;
        } else {
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                const bool ok = x + j < W;
                f0[j] = ok ? feat_in[foff + j] : 0.0f;
                f1[j] = ok ? feat_in[plane + foff + j] : 0.0f;
                f2[j] = ok ? feat_in[2 * plane + foff + j] : 0.0f;
            }
        }
    }

    // Out-of-grid window cells hold a sentinel centre whose D is ~1e18, so
    // the candidate loop needs no bounds checks (the own cell is always
    // valid and always beats it).
    for (int i = tid; i < nwin; i += kThreads) {
        const int qy = i / wnx;
        const int cy = wy0 + qy, cx = wx0 + i - qy * wnx;
        if (cx >= 0 && cx < ns_c && cy >= 0 && cy < ns_r) {
            const float *ck = fa.centres + ((size_t)cy * ns_c + cx) * 6;
            cA[i] = make_float4(ck[0], ck[1], ck[2], ck[3]);
            cY[i] = ck[4];
        } else {
            cA[i] = make_float4(kSentinel, kSentinel, kSentinel, kSentinel);
            cY[i] = kSentinel;
        }
    }
    if (!LAST && !direct) {
        for (int i = tid; i < kWarps * nwin * 4; i += kThreads) {
            const int q = i / (nwin * 4);
            wacc[q * win_max * 4 + (i - q * nwin * 4)] = 0u;
        }
    }
    __syncthreads();

    if (FIRST && row_ok) {
        unsigned r[kPPT], g[kPPT], b[kPPT];
        if (fa.rgb_vec && C == 3) {
            const uint32_t w0 = rgbw[0], w1 = rgbw[1], w2 = rgbw[2];
            r[0] = w0 & 255; g[0] = (w0 >> 8) & 255; b[0] = (w0 >> 16) & 255; r[1] = w0 >> 24;
            g[1] = w1 & 255; b[1] = (w1 >> 8) & 255; r[2] = (w1 >> 16) & 255; g[2] = w1 >> 24;
            b[2] = w2 & 255; r[3] = (w2 >> 8) & 255; g[3] = (w2 >> 16) & 255; b[3] = w2 >> 24;
        } else if (fa.rgb_vec) {
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                r[j] = rgbw[j] & 255; g[j] = (rgbw[j] >> 8) & 255; b[j] = (rgbw[j] >> 16) & 255;
            }
        } else {
            const uint8_t *p = fa.rgb + ((size_t)y * W + x) * C;
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                const bool ok = x + j < W;
                r[j] = ok ? p[j * C + 0] : 0;
                g[j] = ok ? p[j * C + 1] : 0;
                b[j] = ok ? p[j * C + 2] : 0;
            }
        }
#pragma unroll
        for (int j = 0; j < kPPT; ++j) convert_pixel(fa.conv, r[j], g[j], b[j], lut, f0[j], f1[j], f2[j]);
        if (!LAST || store_feat) {
            if ((P & 3) == 0) {
                *reinterpret_cast<float4 *>(feat_out + foff) = make_float4(f0[0], f0[1], f0[2], f0[3]);
                *reinterpret_cast<float4 *>(feat_out + plane + foff) = make_float4(f1[0], f1[1], f1[2], f1[3]);
                *reinterpret_cast<float4 *>(feat_out + 2 * plane + foff) = make_float4(f2[0], f2[1], f2[2], f2[3]);
            } else {
                for (int j = 0; j < kPPT && x + j < W; ++j) {
                    feat_out[foff + j] = f0[j];
                    feat_out[plane + foff + j] = f1[j];
                    feat_out[2 * plane + foff + j] = f2[j];
                }
            }
        }
    }

    // Own cell of each pixel: column cx[j], row pcy.
    const int pcy = div_s(y, s_mul, S);
    int cx[kPPT];
    {
        const int c0 = div_s(x, s_mul, S);
        if (SAME) {
#pragma unroll
            for (int j = 0; j < kPPT; ++j) cx[j] = c0;
        } else if (S >= kPPT) {
            const int rem = x - c0 * S;
#pragma unroll
            for (int j = 0; j < kPPT; ++j) cx[j] = c0 + (rem + j >= S ? 1 : 0);
        } else {
#pragma unroll
            for (int j = 0; j < kPPT; ++j) cx[j] = (x + j) / S;
        }
    }

    // Eq. (1) over the nine centres of the pixel's 3x3 cell window. The
    // candidate's scan position t (dy outer, dx inner) replaces the low 4
    // bits of D (D >= 0, so its bits order like unsigned integers) and one
    // integer min picks the winner: the smallest D, ties to the first in scan
    // order. Values closer than 2^-19 relative also go to scan order.
    unsigned bk[kPPT];
#pragma unroll
    for (int j = 0; j < kPPT; ++j) bk[j] = 0xFFFFFFFFu;
    if (row_ok) {
        const float w = fa.w;
        const float fy = (float)y;
        float fxs[kPPT];
#pragma unroll
        for (int j = 0; j < kPPT; ++j) fxs[j] = (float)(x + j);
        const int rowoff = (pcy - wy0) * wnx - wx0;
#pragma unroll
        for (int jj = 0; jj < (SAME ? 1 : kPPT); ++jj) {
            const int own = rowoff + cx[jj];
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int wi = own + (t / 3 - 1) * wnx + (t % 3 - 1);
                const float4 c = cA[wi];
                const float ddy = cY[wi] - fy;
                const float ddy2 = ddy * ddy;
#pragma unroll
                for (int j = (SAME ? 0 : jj); j < (SAME ? kPPT : jj + 1); ++j) {
                    const float ddx = c.w - fxs[j];
                    const float dl = c.x - f0[j], da = c.y - f1[j], db = c.z - f2[j];
                    const float d_lab = fsqrt_approx(fmaf(dl, dl, fmaf(da, da, db * db)));
                    const float D = fmaf(w, fsqrt_approx(fmaf(ddx, ddx, ddy2)), d_lab);
                    bk[j] = min(bk[j], (__float_as_uint(D) & ~15u) | c_tags[t]);
                }
            }
        }
    }
    // best[j]: the winner as a label (LAST) or as a window index; -1 for
    // pixels outside the image.
    int best[kPPT];
#pragma unroll
    for (int j = 0; j < kPPT; ++j) {
        const int t = (int)(bk[j] & 15u);
        const int dy = t / 3 - 1, dx = t % 3 - 1;
        const bool ok = row_ok && (x + j < W);
        if (LAST)
            best[j] = ok ? (pcy + dy) * ns_c + cx[j] + dx : -1;
        else
            best[j] = ok ? (pcy + dy - wy0) * wnx + (cx[j] + dx - wx0) : -1;
    }

    if constexpr (LAST) {
        if (row_ok) {
            int32_t *out = fa.labels + (size_t)y * W + x;
            if (fa.labels_vec) {
                *reinterpret_cast<int4 *>(out) = make_int4(best[0], best[1], best[2], best[3]);
            } else {
                for (int j = 0; j < kPPT && x + j < W; ++j) out[j] = best[j];
            }
        }
    } else {
        // Partial update sums of this tile. Each lane merges runs of equal
        // choices among its kPPT pixels and adds each run to its warp's
        // private accumulators with four shared-memory atomics: the three
        // feature sums (fixed point) and one word packing the x and y
        // offsets from the tile origin and the count (a warp covers 128
        // pixels, so the fields stay below 2^12, 2^12 and 2^8).
        const float fs = fa.fix_scale;
        if (!direct) {
            unsigned v[kPPT][4];
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                v[j][0] = (unsigned)__float2int_rn(f0[j] * fs);
                v[j][1] = (unsigned)__float2int_rn(f1[j] * fs);
                v[j][2] = (unsigned)__float2int_rn(f2[j] * fs);
                v[j][3] = (unsigned)(x + j - tx0) + ((unsigned)(y - ty0) << 12) + (1u << 24);
            }
#pragma unroll
            for (int j = kPPT - 2; j >= 0; --j) {
                if (best[j + 1] == best[j]) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) v[j][c] += v[j + 1][c];
                }
            }
            unsigned *my = wacc + (size_t)warp * win_max * 4;
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                const int k = (j == 0 || best[j] != best[j - 1]) ? best[j] : -1;
                if (k >= 0) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) atomicAdd(&my[k * 4 + c], v[j][c]);
                }
            }
            __syncthreads();
            // One thread per (window centre, word): add up the 8 warps in
            // int64 and flush to the global sums.
            for (int i = tid; i < nwin * 4; i += kThreads) {
                const int wi = i >> 2, c = i & 3;
                const int qy = wi / wnx;
                const int cy = wy0 + qy, cxg = wx0 + wi - qy * wnx;
                unsigned long long *g =
                    reinterpret_cast<unsigned long long *>(fa.acc) + ((size_t)cy * ns_c + cxg) * 6;
                if (c < 3) {
                    long long t = 0;
#pragma unroll
                    for (int q = 0; q < kWarps; ++q) t += (int)wacc[(size_t)q * win_max * 4 + i];
                    if (t != 0) atomicAdd(&g[c], (unsigned long long)t);
                } else {
                    long long xs = 0, ys = 0, n = 0;
#pragma unroll
                    for (int q = 0; q < kWarps; ++q) {
                        const unsigned pk = wacc[(size_t)q * win_max * 4 + i];
                        xs += pk & 0xFFFu;
                        ys += (pk >> 12) & 0xFFFu;
                        n += pk >> 24;
                    }
                    if (n != 0) {
                        atomicAdd(&g[3], (unsigned long long)(xs + n * tx0));
                        atomicAdd(&g[4], (unsigned long long)(ys + n * ty0));
                        atomicAdd(&g[5], (unsigned long long)n);
                    }
                }
            }
        } else {
            // Very small S: the window is too large for private
            // accumulators; reduce equal keys across the warp and add them to
            // the global sums directly.
            int v[kPPT][6];
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                v[j][0] = __float2int_rn(f0[j] * fs);
                v[j][1] = __float2int_rn(f1[j] * fs);
                v[j][2] = __float2int_rn(f2[j] * fs);
                v[j][3] = x + j;
                v[j][4] = y;
                v[j][5] = 1;
            }
            accumulate_runs(best, v, reinterpret_cast<unsigned long long *>(fa.acc), wx0, wy0, wnx, ns_c);
        }
    }
}

// A middle pass (it accumulates the next update's sums) has nothing to do
// for a frame that passed its stopping test; the last pass always runs.
__device__ __forceinline__ bool frame_stopped(const FrameArgs &a) {
    return a.cstate && a.conv_eps > 0.0f && *reinterpret_cast<const volatile int *>(&a.cstate->done);
}

template <bool FIRST, bool LAST, bool SAME>
__global__ void __launch_bounds__(kThreads, 3) k_assign(const __grid_constant__ FrameArgs a, int store_feat) {
    if (!LAST && frame_stopped(a)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *lut = nullptr;
    if (FIRST) {
        lut = reinterpret_cast<float *>(smem_raw + smem_layout(a.win_max, false));
        for (int i = threadIdx.x; i < 256; i += kThreads) lut[i] = g_lut[i];
    }
    assign_tile<FIRST, LAST, SAME>(a, blockIdx.x * kTileW, blockIdx.y * kTileH, store_feat, smem_raw, lut);
}

// Persistent batched pass: CTA b processes tiles b, b + gridDim.x, ... of
// the concatenated tile lists of all frames (win_max: largest window of any
// frame, which sizes the shared memory).
template <bool FIRST, bool LAST, bool SAME>
__global__ void __launch_bounds__(kThreads, 3) k_assign_batch(const FrameArgs *frames, int n_frames, int total_tiles,
                                                              int win_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *lut = nullptr;
    if (FIRST) {
        lut = reinterpret_cast<float *>(smem_raw + smem_layout(win_max, false));
        for (int i = threadIdx.x; i < 256; i += kThreads) lut[i] = g_lut[i];
    }
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const int f = find_frame<kTileBase>(frames, n_frames, tile);
        const FrameArgs &a = frames[f];
        if (!LAST && frame_stopped(a)) continue;  // CTA-uniform
        const int local = tile - a.tile_base;
        const int ty = local / a.tiles_x, tx = local - ty * a.tiles_x;
        assign_tile<FIRST, LAST, SAME>(a, tx * kTileW, ty * kTileH, 0, smem_raw, lut);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Pipelined assignment for the passes after the first (batched path)
// ---------------------------------------------------------------------------
//
// Persistent CTAs walk the batch's tiles (32 columns by TH = 32 or 64 rows)
// through 3 or 4 shared-memory stages. While the warps evaluate tile i, one
// thread has already issued the two tensor-map copies of the next tiles
// (cp.async.bulk.tensor, completion counted on the stage's mbarrier): the
// 32xTHx3 box of features and the box of 48-byte centre records around the
// tile from the frame's padded centre table (its sentinel ring makes every
// window in-bounds). Lane l of a warp evaluates the 4 pixels at column
// 4*(l%8) of row l/8 of each of its row groups (rows 4w..4w+3 with one row
// group per warp, 8w..8w+3 and 8w+4..8w+7 with two), so each quarter-warp
// reads one 128-byte row without bank conflicts. Stage reuse, the private
// per-tile sums and their flush to the global sums are ordered by mbarriers
// alone: there is no CTA-wide barrier inside the tile loop.

namespace {

__host__ __device__ constexpr size_t stage_feat_bytes(int th) { return (size_t)3 * th * kTileW * 4; }
constexpr int kMaxStages = 4;
constexpr int kAccSets = 2;    // accumulator sets in flight: one filled while the other is flushed
constexpr int kHdrSlots = 8;   // tile-header ring (>= stages + 2)
constexpr unsigned kWaitPolls = 1u << 20;                         // x 1 us suspend hint: ~1 s bound

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Fault injection for tests of the timeout reporting: while non-zero, the
// pipelined assignment's producers issue no further copy (checked before
// each one, so a CTA that gives up has none in flight); the consumers'
// bounded waits then run out.
__device__ int g_abort_copies = 0;

// Wait for the phase with the given parity to complete; gives up (returns
// false) after kWaitPolls polls with a 1 us suspend hint each.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    for (unsigned i = 0; i < kWaitPolls; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity), "r"(1000u)
            : "memory");
        if (done) return true;
    }
    return false;
}


// Paired FP32 arithmetic: a 64-bit operand holds two floats (low, high);
// each element is rounded exactly as the scalar instruction would be.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// min of two non-negative floats (a NaN operand loses), IEEE (no flush).
__device__ __forceinline__ float fmin_nan(float a, float b) {
    float r;
    asm("min.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
// The same over three operands (one instruction on sm_100 and later).
__device__ __forceinline__ float fmin3_nan(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// round(x * fs) (nearest, ties to even) for two values with one paired
// fused multiply-add on the FMA pipe, as a biased word: with M = 1.5 * 2^23,
// x * fs + M lies in [2^23, 2^24) where the float spacing is 1, so the one
// rounding of the fused multiply-add is the rounding to an integer, and the
// float's bits are that integer + kFixBias (the bits of M). Exact for
// |x * fs| < 2^22 (features below 128 at the 2^15 colour scale, 8-bit values
// at scale 1), and equal to __float2int_rn(x * fs) + kFixBias there since fs
// is a power of two. Sums of such words taken mod 2^32, minus count *
// kFixBias, are the sums of the rounded values, exactly, whenever those fit
// in 31 bits (at most 2^22 per value, 128 values per private copy).
constexpr unsigned kFixBias = 0x4B400000u;
__device__ __forceinline__ void fix_round2_biased(float x0, float x1, float fs, unsigned &r0, unsigned &r1) {
    const unsigned long long m = fma2(pack2(x0, x1), pack2(fs, fs), pack2(12582912.0f, 12582912.0f));
    float m0, m1;
    unpack2(m, m0, m1);
    r0 = __float_as_uint(m0);
    r1 = __float_as_uint(m1);
}

// Eq. (1) for two pixels (colour pairs l, a, b; column pair x) against one
// centre record: d_lab = sqrt(dl^2 + da^2 + db^2), d_xy = sqrt(dx^2 + dy^2),
// D = (m/S) d_xy + d_lab, as the two pixels' keys (D & ~15) | t.
__device__ __forceinline__ void eval_keys(const ulonglong2 &la, const ulonglong2 &bx, unsigned long long ddy2,
                                          unsigned long long ww, unsigned long long l, unsigned long long a,
                                          unsigned long long b, unsigned long long x, unsigned t, float &k0,
                                          float &k1) {
    const unsigned long long dl = sub2(la.x, l), da = sub2(la.y, a), db = sub2(bx.x, b);
    const unsigned long long s = fma2(dl, dl, fma2(da, da, mul2(db, db)));
    const unsigned long long dx = sub2(bx.y, x);
    const unsigned long long q = fma2(dx, dx, ddy2);
    float s0, s1, q0, q1;
    unpack2(s, s0, s1);
    unpack2(q, q0, q1);
    const unsigned long long D = fma2(ww, pack2(fsqrt_approx(q0), fsqrt_approx(q1)),
                                      pack2(fsqrt_approx(s0), fsqrt_approx(s1)));
    float d0, d1;
    unpack2(D, d0, d1);
    k0 = __uint_as_float((__float_as_uint(d0) & ~15u) | t);
    k1 = __uint_as_float((__float_as_uint(d1) & ~15u) | t);
}

// Tile header written by the tile's producer next to its stage: the tile's
// geometry and the frame constants the consumers need, so that a warp reads
// one shared-memory record per tile instead of the frame table in global
// memory.
struct __align__(16) TileGeom {
    int tx0, ty0, wx0, wy0;
    int wnx, wny;
    unsigned wnx_mul;      // ceil(2^32 / wnx): cell / wnx for the flush
    int f;                 // frame index
    int W, H, S, ns_c;
    unsigned s_mul;
    int box_w;
    float w, fix_scale;
    int32_t *labels;
    long long *acc;
    int labels_vec;
    int skip;              // 1: the frame passed its stopping test (no copy was issued)
};

// What the fused multi-pass assignment adds to an item's header (a ring of
// its own, beside the tile headers): the item's kind (0: a tile; 1: an
// update chunk, centres c0 .. c0+cn-1 of frame TileGeom::f), its pass (the
// chunk's update is pass + 1) and, for a tile, its frame's counter of
// flushed tiles.
struct MultiHdr {
    int kind, pass, c0, cn;
    int *done_ctr;
};

template <int TH>
__device__ __forceinline__ TileGeom tile_geom(const FrameArgs &a, int local) {
    TileGeom g;
    g.W = a.W;
    g.H = a.H;
    g.S = a.S;
    g.ns_c = a.ns_c;
    g.s_mul = a.s_mul;
    g.box_w = a.box_w;
    g.w = a.w;
    g.fix_scale = a.fix_scale;
    g.labels = a.assign_out;
    g.acc = a.acc;
    g.labels_vec = a.assign_vec;
    g.skip = 0;
    const int ty = local / a.tiles_x, tx = local - ty * a.tiles_x;
    g.tx0 = tx * kTileW;
    g.ty0 = ty * TH;
    const int ccx0 = div_s(g.tx0, a.s_mul, a.S), ccx1 = div_s(min(g.tx0 + kTileW - 1, a.W - 1), a.s_mul, a.S);
    const int ccy0 = div_s(g.ty0, a.s_mul, a.S), ccy1 = div_s(min(g.ty0 + TH - 1, a.H - 1), a.s_mul, a.S);
    g.wx0 = ccx0 - 1;
    g.wy0 = ccy0 - 1;
    g.wnx = ccx1 - ccx0 + 3;
    g.wny = ccy1 - ccy0 + 3;
    g.wnx_mul = (unsigned)((0x100000000ULL + (unsigned)g.wnx - 1) / (unsigned)g.wnx);
    return g;
}

// One thread: arm the stage's mbarrier with the byte count of both boxes
// and issue the two tensor copies.
template <int TH>
__device__ __forceinline__ void issue_tile(const FrameArgs &a, const TileGeom &g, unsigned char *stage,
                                           uint64_t *bar) {
    const unsigned cen_bytes = (unsigned)a.box_w * (unsigned)(TH == 64 ? a.box_h64 : a.box_h) * (unsigned)(kCtabRec * 4);
    mbar_expect_tx(bar, (unsigned)stage_feat_bytes(TH) + cen_bytes);
    tma_load_3d(stage, TH == 64 ? &a.feat_map64 : &a.feat_map, g.tx0, g.ty0, 0, bar);
    tma_load_2d(stage + stage_feat_bytes(TH), TH == 64 ? &a.ctab_map64 : &a.ctab_map, (g.wx0 + 1) * kCtabRec,
                g.wy0 + 1, bar);
}

// Add tile j's private sums (the NCOPY copies of accumulator set j % 2, one
// per 128 pixels) to the frame's global sums and clear them. One of the NW
// warps per tile does it (warp j % NW, so the duty rotates), a lane per
// window cell reading the cell's four words of every copy as one 16-byte
// load. The flushing warp waits
// until every warp has filled the set and reports it free afterwards; the
// others return at once. False when the wait timed out.
template <int NW, int NCOPY, bool MULTI>
__device__ __forceinline__ bool flush_tile(const TileGeom *hdr, const MultiHdr *mhdr, unsigned *wacc0,
                                           size_t acc_words, int win_max, uint64_t *acc_done, uint64_t *acc_free,
                                           int j, int warp, int lane) {
    if (warp != j % NW) return true;
    const int set = j % kAccSets;
    if (!__all_sync(0xffffffffu, mbar_wait(&acc_done[set], (j / kAccSets) & 1))) return false;
    const TileGeom &g = hdr[j % kHdrSlots];
    const int bw = g.box_w, ns_c = g.ns_c, wnx = g.wnx, wny = g.wny, wx0 = g.wx0, wy0 = g.wy0, tx0 = g.tx0,
              ty0 = g.ty0;
    const unsigned wnx_mul = g.wnx_mul;
    long long *const acc = g.acc;
    unsigned *const ws = wacc0 + (size_t)set * acc_words;
    const int n_cells = wnx * wny;
    for (int cell = lane; cell < n_cells; cell += 32) {
        const int qy = (int)__umulhi((unsigned)cell, wnx_mul), qx = cell - qy * wnx;
        const int idx = (qy * bw + qx) * 4;
        long long l = 0, a = 0, b = 0;
        unsigned xs = 0, ys = 0, n = 0;
        // Copies two at a time: the colour words carry kFixBias per pixel
        // (fix_round2_biased), so a pair's words summed mod 2^32 minus its
        // pixel count times kFixBias is the pair's signed sum, exact in 32
        // bits (at most 256 pixels of at most 2^22 each); one 64-bit add per
        // pair and channel. Copy q's y field counts from the tile's first row
        // (32-row tiles) or from its warp's first row, 8 (q / 2) (64-row
        // tiles, whose offsets would not fit the 12-bit field).
        static_assert(NCOPY % 2 == 0, "copies are summed in pairs");
#pragma unroll
        for (int q = 0; q < NCOPY; q += 2) {
            uint4 *p0 = reinterpret_cast<uint4 *>(ws + (size_t)q * win_max * 4 + idx);
            uint4 *p1 = reinterpret_cast<uint4 *>(ws + (size_t)(q + 1) * win_max * 4 + idx);
            const uint4 v0 = *p0, v1 = *p1;
            *p0 = make_uint4(0u, 0u, 0u, 0u);
            *p1 = make_uint4(0u, 0u, 0u, 0u);
            const unsigned n0 = v0.w >> 24, n1 = v1.w >> 24;
            const unsigned bias = (n0 + n1) * kFixBias;
            l += (int)(v0.x + v1.x - bias);
            a += (int)(v0.y + v1.y - bias);
            b += (int)(v0.z + v1.z - bias);
            xs += (v0.w & 0xFFFu) + (v1.w & 0xFFFu);
            ys += ((v0.w >> 12) & 0xFFFu) + ((v1.w >> 12) & 0xFFFu) +
                  (NCOPY > kWarps ? 8u * (unsigned)(q >> 1) * (n0 + n1) : 0u);
            n += n0 + n1;
        }
        if (n != 0) {
            unsigned long long *gs =
                reinterpret_cast<unsigned long long *>(acc) + ((size_t)(wy0 + qy) * ns_c + wx0 + qx) * 6;
            atomicAdd(&gs[0], (unsigned long long)l);
            atomicAdd(&gs[1], (unsigned long long)a);
            atomicAdd(&gs[2], (unsigned long long)b);
            atomicAdd(&gs[3], (unsigned long long)xs + (unsigned long long)n * tx0);
            atomicAdd(&gs[4], (unsigned long long)ys + (unsigned long long)n * ty0);
            atomicAdd(&gs[5], (unsigned long long)n);
        }
    }
    __syncwarp();
    if (lane == 0) {
        if constexpr (MULTI) {
            // the tile's sums are in the frame's global sums: count it (release)
            int *const ctr = mhdr[j % kHdrSlots].done_ctr;
            if (ctr) {
                __threadfence();
                atomicAdd(ctr, 1);
            }
        }
        mbar_arrive(&acc_free[set]);
    }
    return true;
}

// Polls of wait_count: with a 256 ns sleep each, about 1 s in all.
constexpr unsigned kCountPolls = 1u << 22;

// Bounded wait of one thread until the counter at p reaches target (acquire
// at device scope); false when it gives up, or as soon as *err is set.
__device__ __forceinline__ bool wait_count(const int *p, int target, const int *err) {
    for (unsigned i = 0; i < kCountPolls; ++i) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= target) return true;
        if (*reinterpret_cast<const volatile int *>(err)) return false;
        __nanosleep(256);
    }
    return false;
}

// Orders this thread's global accesses of the generic proxy with those of
// the async proxy (the tensor copies): centre records written by one CTA
// are read by another CTA's tensor copy in the same launch.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

}  // namespace

// Member mean from the exact integer sums, in FP32 (this GPU's FP64 rate is
// a small fraction of its FP32 rate): the sum rounded to float, scaled by the
// power of two fix_inv (exact) and divided by the count (correctly rounded),
// so within about one unit in the last place of the exact mean.
// Returns the centre's move |dx| + |dy| (0 for an empty cluster, or when
// want_move is false: the old position is then not read).
__device__ __forceinline__ float update_centre(long long *ak, const float *ci, float *co, float fix_inv,
                                               bool want_move) {
    // (L2 loads: in the fused multi-pass assignment other CTAs wrote these in
    // the same launch)
    const longlong2 s01 = __ldcg(reinterpret_cast<const longlong2 *>(ak));
    const longlong2 s23 = __ldcg(reinterpret_cast<const longlong2 *>(ak + 2));
    const longlong2 s45 = __ldcg(reinterpret_cast<const longlong2 *>(ak + 4));
    const long long n = s45.y;
    float move = 0.0f;
    if (n > 0) {
        const float fn = (float)n;
        const float x0 = want_move ? __ldcg(ci + 3) : 0.0f, y0 = want_move ? __ldcg(ci + 4) : 0.0f;
        co[0] = __fdiv_rn((float)s01.x * fix_inv, fn);
        co[1] = __fdiv_rn((float)s01.y * fix_inv, fn);
        co[2] = __fdiv_rn((float)s23.x * fix_inv, fn);
        const float xn = __fdiv_rn((float)s23.y, fn), yn = __fdiv_rn((float)s45.x, fn);
        co[3] = xn;
        co[4] = yn;
        co[5] = fn;
        if (want_move) move = fabsf(xn - x0) + fabsf(yn - y0);
    } else {
        if (co != ci) {
#pragma unroll
            for (int c = 0; c < 5; ++c) co[c] = __ldcg(ci + c);
        }
        co[5] = 0.0f;
    }
    longlong2 *az = reinterpret_cast<longlong2 *>(ak);
    az[0] = make_longlong2(0, 0);
    az[1] = make_longlong2(0, 0);
    az[2] = make_longlong2(0, 0);
    return move;
}

// Stopping test before update `it` (1-based): the frame stops when it has
// stopped already or update it-1 moved its K centres by a mean L1 distance
// below eps (so update it-1 and its assignment were the last). Every thread
// decides from the same stored values.
__device__ __forceinline__ bool conv_stop(const ConvState *cs, float eps, int K, int it) {
    if (!cs || !(eps > 0.0f)) return false;
    if (*reinterpret_cast<const volatile int *>(&cs->done)) return true;
    if (it < 2) return false;
    long long e = 0;
#pragma unroll
    for (int i = 0; i < kResidLanes; ++i) e += __ldcg(&cs->resid[(it - 1) % 3][i]);
    return (double)e < (double)eps * (double)kResidScale * (double)K;
}

// After update `it`: with the stopping test on, the sum of this warp's
// moves into one of the frame's counters of slot it % 3 (one atomic per
// warp when all its lanes belong to `cs`'s frame); from the frame's first
// centre, the update count and the cleared slot of update it+1.
__device__ __forceinline__ void conv_record(ConvState *cs, bool uniform, bool test_on, float move, bool first,
                                            int it) {
    if (test_on) {
        long long v = (long long)__float2ll_rn(move * kResidScale);
        const int lane_slot = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) % kResidLanes;
        if (uniform) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0 && v != 0)
                atomicAdd(reinterpret_cast<unsigned long long *>(&cs->resid[it % 3][lane_slot]), (unsigned long long)v);
        } else if (v != 0) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&cs->resid[it % 3][lane_slot]), (unsigned long long)v);
        }
    }
    if (first) {
        if (test_on) {
#pragma unroll
            for (int i = 0; i < kResidLanes; ++i) cs->resid[(it + 1) % 3][i] = 0;
        }
        cs->iters = it;
    }
}

size_t assign_pipe_smem_bytes(int win_n, bool last, int nst, int rows, int tile_h, bool multi) {
    (void)rows;  // the sums keep one copy per 128 pixels whatever the warp count
    const size_t stage = stage_feat_bytes(tile_h) + (((size_t)win_n * kCtabRec * 4 + 127) & ~(size_t)127);
    const size_t acc = last ? 0 : (size_t)kWarps * (tile_h / kTileH) * win_n * 4 * sizeof(int);
    // nst stages, the accumulator sets, the mbarriers, the header ring, two
    // flags and base alignment
    return (size_t)nst * stage + kAccSets * acc + (size_t)(2 * kMaxStages + 2 * kAccSets) * 8 +
           (size_t)kHdrSlots * sizeof(TileGeom) + 16 + 128 + (multi ? (size_t)kHdrSlots * sizeof(MultiHdr) : 0);
}

// An update chunk of the fused multi-pass assignment: update `it` of
// centres c0 .. c0+cn-1 of one frame by the CTA's NT threads, as
// k_update_batch does it (stopping test, member means, centre records,
// cleared sums, the frame's move).
template <int NT>
__device__ __forceinline__ void update_chunk(const FrameArgs &a, int c0, int cn, int it, int tid) {
    const int K = a.ns_c * a.ns_r;
    for (int i = 0; i < kUpdateChunk; i += NT) {  // the same trip count on every lane
        const int j = i + tid, kk = c0 + j;
        const bool valid = j < cn;
        float move = 0.0f;
        bool stop = true;
        if (valid) {
            stop = conv_stop(a.cstate, a.conv_eps, K, it);
            if (stop) {
                if (kk == 0) a.cstate->done = 1;
            } else {
                const size_t k = (size_t)kk * 6;
                move = update_centre(a.acc + k, a.centres_out + k, a.centres_out + k, 1.0f / a.fix_scale,
                                     a.conv_eps > 0.0f);
                const int r = kk / a.ns_c, c = kk - r * a.ns_c;
                write_ctab(a.ctab + ((size_t)(r + 1) * (a.ns_c + 2) + c + 1) * kCtabRec, a.centres_out + k);
            }
        }
        // (a frame stops for all its centres: a warp of valid lanes is all
        // stopped or all running)
        if (__all_sync(kFull, valid)) {
            if (!stop) conv_record(a.cstate, true, a.conv_eps > 0.0f, move, kk == 0, it);
        } else if (valid && !stop) {
            conv_record(a.cstate, false, a.conv_eps > 0.0f, move, kk == 0, it);
        }
    }
}

// The pipelined assignment, as one pass (k_assign_pipe) or as the fused
// passes before the last (k_assign_multi, MULTI).
template <bool LAST, bool SAME, int MINB, int ROWS, int TH, bool MULTI>
__device__ __forceinline__ void assign_pipe_body(const FrameArgs *frames, int n_frames, int total_tiles, int win_max,
                                                 int nst, int *err, int check_stop, int passes, int total_chunks) {
    // ROWS = 1: 8 warps, warp w evaluates rows 4w..4w+3 of the tile.
    // ROWS = 2: TH/8 warps, warp w evaluates rows 8w..8w+3 and 8w+4..8w+7
    // (the same cell row when S is a multiple of 8), sharing the centre loads
    // and the per-tile work between 8 pixels per thread. TH: tile rows (32,
    // or 64 with ROWS = 2).
    static_assert(ROWS == 1 || (ROWS == 2 && SAME), "two row groups need cell-aligned 4-pixel groups");
    static_assert(TH == 32 || (TH == 64 && ROWS == 2), "32x64 tiles with two row groups only");
    static_assert(!(MULTI && LAST), "the fused passes accumulate sums; the last pass is a launch of its own");
    constexpr int NW = kWarps / ROWS * (TH / 32), NT = NW * 32;
    constexpr int NCOPY = NW * ROWS;  // private sums: one copy per 128 pixels (rows 4q .. 4q+3)
    constexpr size_t kFeat = stage_feat_bytes(TH);
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    // Tensor copies want 128-byte aligned destinations.
    unsigned char *smem_raw =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~(uintptr_t)127);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t stage_bytes = kFeat + (((size_t)win_max * kCtabRec * 4 + 127) & ~(size_t)127);
    // One private copy of the sums per 128 pixels (per warp and row group),
    // so a copy's packed x / y / count fields cannot overflow.
    const size_t acc_words = LAST ? 0 : (size_t)NCOPY * win_max * 4;
    unsigned *const wacc0 = reinterpret_cast<unsigned *>(smem_raw + (size_t)nst * stage_bytes);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)nst * stage_bytes + kAccSets * acc_words * 4);
    uint64_t *empty = full + kMaxStages;       // stage released by every warp (count NW)
    uint64_t *acc_done = empty + kMaxStages;   // accumulator set filled by every warp (count NW)
    uint64_t *acc_free = acc_done + kAccSets;  // accumulator set flushed and cleared (count 1)
    TileGeom *hdr = reinterpret_cast<TileGeom *>(acc_free + kAccSets);  // ring of kHdrSlots tile headers
    int *flags = reinterpret_cast<int *>(hdr + kHdrSlots);              // [0] abort, [1] last tile issued
    MultiHdr *mhdr = reinterpret_cast<MultiHdr *>(flags + 4);           // MULTI: ring of kHdrSlots records
    volatile int *abort_flag = flags;
    const int ahead = nst - 3;  // tiles issued beyond the next one: stage reuse lags two tiles
    // Work items of this CTA. One pass: tiles blockIdx.x + i * gridDim.x of
    // the batch. MULTI, in every pass: a contiguous block of the batch's
    // tiles (frame after frame), tiles t_lo .. t_lo+n_t-1, then the same
    // share of its update chunks, k_lo .. k_lo+n_k-1 (blocks of CTA c:
    // [c*N/G, (c+1)*N/G)); item j is item j % n_local of pass j / n_local.
    int n_local, t_lo = 0, n_t = 0, k_lo = 0;
    if constexpr (MULTI) {
        const long long G = gridDim.x, c = blockIdx.x;
        t_lo = (int)(total_tiles * c / G);
        n_t = (int)(total_tiles * (c + 1) / G) - t_lo;
        k_lo = (int)(total_chunks * c / G);
        n_local = n_t + (int)(total_chunks * (c + 1) / G) - k_lo;
    } else {
        n_local = (int)blockIdx.x < total_tiles
                      ? (total_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                      : 0;
    }
    const int n_items = MULTI ? n_local * passes : n_local;

    if (tid == 0) {
        for (int q = 0; q < nst; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], NW);
        }
        for (int q = 0; q < kAccSets; ++q) {
            mbar_init(&acc_done[q], NW);
            mbar_init(&acc_free[q], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        flags[0] = 0;
        flags[1] = -1;
    }
    if (!LAST) {
        for (int i = tid; i < (int)(kAccSets * acc_words); i += NT) wacc0[i] = 0u;
    }
    __syncthreads();

    // Item j of this CTA goes to stage j % nst (its use j / nst of that
    // stage) and header slot j % kHdrSlots. Its producer issues it at the top
    // of iteration j - ahead - 1, once every warp has released the stage's
    // previous item j - nst (two iterations earlier); the producer role
    // rotates over the warps. No CTA-wide barrier inside the loop: warps
    // drift up to about two items apart, bounded by the mbarriers.
    // q = j % nst and use = j / nst are passed in (kept incrementally: a
    // division by the run-time stage count costs tens of instructions).
    //
    // MULTI: an update chunk waits (bounded) until its frame's tiles of the
    // pass are all in the global sums; a tile of pass p > 0 is issued once
    // every chunk of its frame's update p is done. The CTAs sharing a frame's
    // tiles share its chunks, so a frame's waits involve those CTAs only.
    // Each wait is on items of an earlier level (pass, tiles before chunks),
    // and a CTA waits only when its own items of earlier levels are
    // finished: it flushes the previous item before a chunk waits, flushes a
    // pass's last item at once, and issues no item of the next pass before
    // that flush (no look-ahead across passes). With every CTA resident (a
    // cooperative launch) the items of the earliest unfinished level can
    // always proceed, so every wait ends.
    // MULTI: the (frame, pass) whose dependency this producer thread last
    // verified; its later tiles of the same frame and pass need no new check
    // (the condition only becomes true once, and this thread's acquire and
    // proxy fence precede all its later copies).
    int dep_f = -1, dep_pass = -1;
    int pf = 0;  // frame of this producer thread's last tile (one launch per pass)
    auto produce = [&](int j, int q, int use) -> bool {
        if constexpr (MULTI) {
            if (j >= n_items) return true;
            if (*reinterpret_cast<volatile int *>(&g_abort_copies)) return false;
            if (use > 0 && !mbar_wait(&empty[q], (use - 1) & 1)) return false;
            const int pass = j / n_local;
            const int i = j - pass * n_local;
            MultiHdr m;
            m.pass = pass;
            if (i < n_t) {
                const int t = t_lo + i;
                const int f = find_frame<TH == 64 ? kTileBase64 : kTileBase>(frames, n_frames, t);
                if (pass > 0 && (f != dep_f || pass != dep_pass)) {
                    if (!wait_count(&frames[f].cstate->chunks_done, frames[f].n_chunks * NW * pass, err))
                        return false;
                    fence_proxy_async_global();  // the chunks' centre records, before the tensor copy
                    dep_f = f;
                    dep_pass = pass;
                }
                TileGeom g = tile_geom<TH>(frames[f], t - base_of<TH == 64 ? kTileBase64 : kTileBase>(frames[f]));
                g.f = f;
                g.skip = check_stop && frame_stopped(frames[f]) ? 1 : 0;
                if (g.skip) g.H = 0;  // no pixel of the tile is evaluated or summed
                m.kind = 0;
                m.c0 = m.cn = 0;
                m.done_ctr = &frames[f].cstate->tiles_done;
                hdr[j % kHdrSlots] = g;
                mhdr[j % kHdrSlots] = m;
                if (g.skip)
                    mbar_arrive(&full[q]);
                else
                    issue_tile<TH>(frames[f], g, smem_raw + (size_t)q * stage_bytes, &full[q]);
            } else {
                const int k = k_lo + (i - n_t);
                const int f = find_frame<kChunkBase>(frames, n_frames, k);
                TileGeom g = TileGeom{};
                g.f = f;
                m.kind = 1;
                m.c0 = (k - frames[f].chunk_base) * kUpdateChunk;
                m.cn = min(kUpdateChunk, frames[f].ns_c * frames[f].ns_r - m.c0);
                m.done_ctr = nullptr;
                hdr[j % kHdrSlots] = g;
                mhdr[j % kHdrSlots] = m;
                mbar_arrive(&full[q]);  // no data: the stage completes at once
            }
            atomicMax(&flags[1], j);
            return true;
        } else {
            const int t = blockIdx.x + j * gridDim.x;
            if (t >= total_tiles) return true;
            if (*reinterpret_cast<volatile int *>(&g_abort_copies)) return false;
            if (use > 0 && !mbar_wait(&empty[q], (use - 1) & 1)) return false;
            // A producer thread's tiles come in increasing order: its frame
            // index only moves forward.
            while (pf + 1 < n_frames && base_of<TH == 64 ? kTileBase64 : kTileBase>(frames[pf + 1]) <= t) ++pf;
            const int f = pf;
            TileGeom g = tile_geom<TH>(frames[f], t - base_of<TH == 64 ? kTileBase64 : kTileBase>(frames[f]));
            g.f = f;
            g.skip = !LAST && check_stop && frame_stopped(frames[f]) ? 1 : 0;
            if (g.skip) g.H = 0;  // no pixel of the tile is evaluated or summed
            hdr[j % kHdrSlots] = g;
            if (g.skip)
                mbar_arrive(&full[q]);  // a stopped frame's tile: no copy, the stage completes at once
            else
                issue_tile<TH>(frames[f], g, smem_raw + (size_t)q * stage_bytes, &full[q]);
            atomicMax(&flags[1], j);
            return true;
        }
    };
    if (tid == 0) {
        for (int j = 0; j <= ahead && (!MULTI || j < n_local); ++j) produce(j, j, 0);
    }
    __syncthreads();
    // Stage and phase of this iteration's tile, and of the tile its producer
    // issues (ahead + 1 later), advanced without division.
    int s = 0, ph = 0, sp = ahead + 1, usep = 0;
    if (sp == nst) {
        sp = 0;
        usep = 1;
    }

    const int lx = 4 * (lane & 7), ly0 = 4 * ROWS * warp + (lane >> 3);
    int it = 0;
    bool ok = true;
    // MULTI: position of item `it` in its pass, the CTA's first item of the
    // next pass, and whether item it-1 closed a pass (it was flushed then)
    int pit = 0, pass_end = n_local;
    bool prev_flushed = false;
    auto advance = [&]() {
        if (++s == nst) {
            s = 0;
            ph ^= 1;
        }
        if (++sp == nst) {
            sp = 0;
            ++usep;
        }
        if constexpr (MULTI) {
            if (++pit == n_local) {
                pit = 0;
                pass_end += n_local;
            }
        }
    };
    for (int tile = blockIdx.x; MULTI ? it < n_items : tile < total_tiles; tile += gridDim.x, ++it, advance()) {
        if (*abort_flag) {
            ok = false;
            break;
        }
        if (warp == it % NW && lane == 0) {
            bool okp = true;
            if constexpr (MULTI) {
                if (pit == 0 && it > 0) {
                    // A new pass: once this CTA's last item of the previous
                    // pass is flushed, the pass's first items (held back)
                    // are issued.
                    okp = mbar_wait(&acc_free[(it - 1) % kAccSets], ((it - 1) / kAccSets) & 1);
                    for (int j = it; okp && j <= it + ahead && j < pass_end; ++j) okp = produce(j, j % nst, j / nst);
                }
                if (okp && it + ahead + 1 < pass_end) okp = produce(it + ahead + 1, sp, usep);
            } else {
                okp = produce(it + ahead + 1, sp, usep);
            }
            if (!okp) {
                *abort_flag = 1;
                atomicOr(err, 1);
            }
        }
        if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph & 1))) {
            if (lane == 0) {
                *abort_flag = 1;
                atomicOr(err, 1);
            }
            ok = false;
            break;
        }
        unsigned char *const stage_s = smem_raw + (size_t)s * stage_bytes;
        const TileGeom &g = hdr[it % kHdrSlots];
        if constexpr (MULTI) {
            const MultiHdr &mh = mhdr[it % kHdrSlots];
            if (mh.kind == 1) {
                // An update chunk: no data in the stage, no pixel sums.
                const int cf = g.f, c0 = mh.c0, cn = mh.cn, cpass = mh.pass;
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
                const int set = it % kAccSets;
                bool okc =
                    it < kAccSets || __all_sync(0xffffffffu, mbar_wait(&acc_free[set], ((it / kAccSets) - 1) & 1));
                // The previous item's sums first: its tile may be one this
                // chunk waits for.
                if (okc && it > 0 && !prev_flushed)
                    okc = flush_tile<NW, NCOPY, MULTI>(hdr, mhdr, wacc0, acc_words, win_max, acc_done, acc_free, it - 1,
                                                       warp, lane);
                const FrameArgs &a = frames[cf];
                if (okc) {
                    bool okw = true;
                    if (lane == 0)
                        okw = wait_count(&a.cstate->tiles_done, (TH == 64 ? a.n_tiles64 : a.n_tiles) * (cpass + 1),
                                         err);
                    okc = __shfl_sync(0xffffffffu, okw ? 1 : 0, 0) != 0;
                }
                if (okc) {
                    update_chunk<NT>(a, c0, cn, cpass + 1, tid);
                    __syncwarp();
                    if (lane == 0) {
                        // this warp's part of the chunk is done (release)
                        fence_proxy_async_global();
                        __threadfence();
                        atomicAdd(&a.cstate->chunks_done, 1);
                        mbar_arrive(&acc_done[set]);
                    }
                    if (pit == n_local - 1)
                        okc = flush_tile<NW, NCOPY, MULTI>(hdr, mhdr, wacc0, acc_words, win_max, acc_done, acc_free, it,
                                                           warp, lane);
                    prev_flushed = pit == n_local - 1;
                }
                if (!okc) {
                    if (lane == 0) {
                        *abort_flag = 1;
                        atomicOr(err, 1);
                    }
                    ok = false;
                    break;
                }
                continue;
            }
        }
        const int bw = g.box_w, tx0 = g.tx0, ty0 = g.ty0, wx0 = g.wx0, wy0 = g.wy0;
        const int W = g.W, H = g.H, S = g.S, ns_c = g.ns_c;
        const unsigned s_mul = g.s_mul;
        const float *feat = reinterpret_cast<const float *>(stage_s);
        const float *cen = reinterpret_cast<const float *>(stage_s + kFeat);
        const int x = tx0 + lx;
        int y[ROWS];
        bool row_ok[ROWS];
        float f0[ROWS][kPPT] = {}, f1[ROWS][kPPT] = {}, f2[ROWS][kPPT] = {};
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int ly = ly0 + 4 * r;
            y[r] = ty0 + ly;
            row_ok[r] = (y[r] < H) && (x < W);  // (H = 0 in a skipped tile's header)
            if (row_ok[r]) {
                const float4 v0 = *reinterpret_cast<const float4 *>(feat + (0 * TH + ly) * kTileW + lx);
                const float4 v1 = *reinterpret_cast<const float4 *>(feat + (1 * TH + ly) * kTileW + lx);
                const float4 v2 = *reinterpret_cast<const float4 *>(feat + (2 * TH + ly) * kTileW + lx);
                f0[r][0] = v0.x; f0[r][1] = v0.y; f0[r][2] = v0.z; f0[r][3] = v0.w;
                f1[r][0] = v1.x; f1[r][1] = v1.y; f1[r][2] = v1.z; f1[r][3] = v1.w;
                f2[r][0] = v2.x; f2[r][1] = v2.y; f2[r][2] = v2.z; f2[r][3] = v2.w;
            }
        }
        // Both row groups share the cell row (ROWS = 2 needs S % 8 == 0).
        const int pcy = div_s(y[0], s_mul, S);
        int cx[kPPT];
        {
            const int c0 = div_s(x, s_mul, S);
            if (SAME) {
#pragma unroll
                for (int j = 0; j < kPPT; ++j) cx[j] = c0;
            } else if (S >= kPPT) {
                const int rem = x - c0 * S;
#pragma unroll
                for (int j = 0; j < kPPT; ++j) cx[j] = c0 + (rem + j >= S ? 1 : 0);
            } else {
#pragma unroll
                for (int j = 0; j < kPPT; ++j) cx[j] = (x + j) / S;
            }
        }
        // Eq. (1) over the nine window centres, as in assign_tile (window
        // index = (cell row - wy0) * box_w + (cell column - wx0)), with the
        // same operations in the same order. The running minimum is a float
        // whose low 4 mantissa bits carry the candidate index: non-negative
        // floats order like their bit patterns, so this equals the integer
        // minimum of (D & ~15) | t, scan order breaking ties.
        float bk[ROWS][kPPT];
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
#pragma unroll
            for (int j = 0; j < kPPT; ++j) bk[r][j] = __int_as_float(0x7F800000);
        bool any_row = false;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) any_row |= row_ok[r];
        if (any_row) {
            const float w = g.w;
            const int rowoff = (pcy - wy0) * bw - wx0;
            if (SAME) {
                // The thread's pixels share the window: pixels (0, 1) and
                // (2, 3) of each row group go through paired FP32 instructions.
                const unsigned long long ww = pack2(w, w);
                unsigned long long fyy[ROWS], l01[ROWS], l23[ROWS], a01[ROWS], a23[ROWS], b01[ROWS], b23[ROWS];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const float fy = (float)y[r];
                    fyy[r] = pack2(fy, fy);
                    l01[r] = pack2(f0[r][0], f0[r][1]);
                    l23[r] = pack2(f0[r][2], f0[r][3]);
                    a01[r] = pack2(f1[r][0], f1[r][1]);
                    a23[r] = pack2(f1[r][2], f1[r][3]);
                    b01[r] = pack2(f2[r][0], f2[r][1]);
                    b23[r] = pack2(f2[r][2], f2[r][3]);
                }
                const float fx = (float)x;  // x + j exactly (x < 2^24)
                const unsigned long long x01 = pack2(fx, fx + 1.0f), x23 = pack2(fx + 2.0f, fx + 3.0f);
                const int own = rowoff + cx[0];
                // Candidates two at a time: each pixel's running minimum takes
                // both keys in one three-operand min (keys are distinct, so
                // the grouping does not change the result).
#pragma unroll
                for (int t0 = 0; t0 < 9; t0 += 2) {
                    const int nt = t0 < 8 ? 2 : 1;
                    float kk[2][ROWS][kPPT];
#pragma unroll
                    for (int u = 0; u < nt; ++u) {
                        const int t = t0 + u;
                        const float *rp = cen + (size_t)(own + (t / 3 - 1) * bw + (t % 3 - 1)) * kCtabRec;
                        const ulonglong2 la = *reinterpret_cast<const ulonglong2 *>(rp);      // (L, L), (a, a)
                        const ulonglong2 bx = *reinterpret_cast<const ulonglong2 *>(rp + 4);  // (b, b), (x, x)
                        const unsigned long long yy = *reinterpret_cast<const unsigned long long *>(rp + 8);
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) {
                            const unsigned long long ddy = sub2(yy, fyy[r]);
                            const unsigned long long ddy2 = mul2(ddy, ddy);
                            eval_keys(la, bx, ddy2, ww, l01[r], a01[r], b01[r], x01, c_tags[t], kk[u][r][0],
                                      kk[u][r][1]);
                            eval_keys(la, bx, ddy2, ww, l23[r], a23[r], b23[r], x23, c_tags[t], kk[u][r][2],
                                      kk[u][r][3]);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < ROWS; ++r)
#pragma unroll
                        for (int j = 0; j < kPPT; ++j)
                            bk[r][j] = nt == 2 ? fmin3_nan(bk[r][j], kk[0][r][j], kk[1][r][j])
                                               : fmin_nan(bk[r][j], kk[0][r][j]);
                }
            } else {
                const float fy = (float)y[0];
#pragma unroll
                for (int j = 0; j < kPPT; ++j) {
                    const int own = rowoff + cx[j];
                    const float fx = (float)(x + j);
#pragma unroll
                    for (int t = 0; t < 9; ++t) {
                        const float *rp = cen + (size_t)(own + (t / 3 - 1) * bw + (t % 3 - 1)) * kCtabRec;
                        const float4 la = *reinterpret_cast<const float4 *>(rp);
                        const float4 bx = *reinterpret_cast<const float4 *>(rp + 4);
                        const float ddy = rp[8] - fy;
                        const float ddx = bx.z - fx;
                        const float dl = la.x - f0[0][j], da = la.z - f1[0][j], db = bx.x - f2[0][j];
                        const float d_lab = fsqrt_approx(fmaf(dl, dl, fmaf(da, da, db * db)));
                        const float D = fmaf(w, fsqrt_approx(fmaf(ddx, ddx, ddy * ddy)), d_lab);
                        bk[0][j] = fmin_nan(bk[0][j], __uint_as_float((__float_as_uint(D) & ~15u) | c_tags[t]));
                    }
                }
            }
        }
        // Winner t -> its cell: row offset t/3 - 1, column offset t%3 - 1, so
        // index = base + t + (t/3)*(stride - 3) with base = own - stride - 1
        // (stride: box_w for the window index of the sums, ns_c for the label).
        int best[ROWS][kPPT];
        {
            const int stride = LAST ? ns_c : bw;
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                const int base = (LAST ? pcy * ns_c + cx[j] : (pcy - wy0) * bw + cx[j] - wx0) - stride - 1;
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const unsigned t = __float_as_uint(bk[r][j]) & 15u;
                    const int q = (int)__umulhi(t, 0x55555556u);  // t / 3 for t < 9
                    const bool okp = row_ok[r] && (x + j < W);
                    best[r][j] = okp ? base + (int)t + q * (stride - 3) : -1;
                }
            }
        }
        // Every read of the stage is done: release it to the producers.
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                if (row_ok[r]) {
                    int32_t *out = g.labels + (size_t)y[r] * W + x;
                    if (g.labels_vec) {
                        *reinterpret_cast<int4 *>(out) = make_int4(best[r][0], best[r][1], best[r][2], best[r][3]);
                    } else {
                        for (int j = 0; j < kPPT && x + j < W; ++j) out[j] = best[r][j];
                    }
                }
            }
        } else {
            const float fs = g.fix_scale;
            // Set it % 2 was flushed (tile it - 2) before it is reused.
            const int set = it % kAccSets;
            if (it >= kAccSets && !__all_sync(0xffffffffu, mbar_wait(&acc_free[set], ((it / kAccSets) - 1) & 1))) {
                if (lane == 0) {
                    *abort_flag = 1;
                    atomicOr(err, 1);
                }
                ok = false;
                break;
            }
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                // One row group: copy q = warp holds rows 4q .. 4q+3. Two row
                // groups: copy q = 2 warp + (lane >> 4), the lanes of one half
                // of the warp in both groups (rows 8 warp + {2h, 2h+1, 2h+4,
                // 2h+5}, h = q % 2), so an instruction's atomics go to two
                // copies and fewer lanes meet on one address. y counts from the
                // tile's first row (32-row tiles) or from the warp's first row
                // (64-row tiles; see flush_tile).
                const int q = ROWS == 2 ? 2 * warp + (lane >> 4) : warp;
                unsigned *my = wacc0 + (size_t)set * acc_words + (size_t)q * win_max * 4;
                unsigned v[kPPT][4];
                const unsigned yo = TH == 64 ? (unsigned)((lane >> 3) + 4 * r) : (unsigned)(ly0 + 4 * r);
                const unsigned xyn = (unsigned)lx + (yo << 12) + (1u << 24);
#pragma unroll
                for (int j = 0; j < kPPT; j += 2) {
                    fix_round2_biased(f0[r][j], f0[r][j + 1], fs, v[j][0], v[j + 1][0]);
                    fix_round2_biased(f1[r][j], f1[r][j + 1], fs, v[j][1], v[j + 1][1]);
                    fix_round2_biased(f2[r][j], f2[r][j + 1], fs, v[j][2], v[j + 1][2]);
                    v[j][3] = xyn + (unsigned)j;
                    v[j + 1][3] = xyn + (unsigned)(j + 1);
                }
#pragma unroll
                for (int j = kPPT - 2; j >= 0; --j) {
                    if (best[r][j + 1] == best[r][j]) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) v[j][c] += v[j + 1][c];
                    }
                }
#pragma unroll
                for (int j = 0; j < kPPT; ++j) {
                    const int k = (j == 0 || best[r][j] != best[r][j - 1]) ? best[r][j] : -1;
                    if (k >= 0) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) atomicAdd(&my[k * 4 + c], v[j][c]);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_done[set]);
            // Flush the previous tile's sums (one warp per tile).
            if (it > 0 && !(MULTI && prev_flushed) &&
                !flush_tile<NW, NCOPY, MULTI>(hdr, mhdr, wacc0, acc_words, win_max, acc_done, acc_free, it - 1, warp,
                                              lane)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    atomicOr(err, 1);
                }
                ok = false;
                break;
            }
            if constexpr (MULTI) {
                // a pass's last item is flushed at once (see above)
                if (pit == n_local - 1 &&
                    !flush_tile<NW, NCOPY, MULTI>(hdr, mhdr, wacc0, acc_words, win_max, acc_done, acc_free, it, warp,
                                                  lane)) {
                    if (lane == 0) {
                        *abort_flag = 1;
                        atomicOr(err, 1);
                    }
                    ok = false;
                    break;
                }
                prev_flushed = pit == n_local - 1;
            }
        }
    }
    if (!LAST && !MULTI && ok && it > 0 &&
        !flush_tile<NW, NCOPY, MULTI>(hdr, mhdr, wacc0, acc_words, win_max, acc_done, acc_free, it - 1, warp, lane)) {
        if (lane == 0) {
            *abort_flag = 1;
            atomicOr(err, 1);
        }
    }
    __syncthreads();
    if (tid == 0 && *abort_flag) {
        // A wait timed out: let the copies already issued land (bounded)
        // before the CTA exits, so none targets freed shared memory.
        const int last = flags[1];
        for (int j = max(0, last - nst + 1); j <= last; ++j) mbar_wait(&full[j % nst], (j / nst) & 1);
    }
}

template <bool LAST, bool SAME, int MINB, int ROWS, int TH>
__global__ void __launch_bounds__(kThreads / ROWS * (TH / 32), MINB)
    k_assign_pipe(const FrameArgs *frames, int n_frames, int total_tiles, int win_max, int nst, int *err,
                  int check_stop) {
    assign_pipe_body<LAST, SAME, MINB, ROWS, TH, false>(frames, n_frames, total_tiles, win_max, nst, err, check_stop,
                                                        1, 0);
}

// The passes before the last with their updates, in one cooperative launch.
template <bool SAME, int MINB, int ROWS, int TH>
__global__ void __launch_bounds__(kThreads / ROWS * (TH / 32), MINB)
    k_assign_multi(const FrameArgs *frames, int n_frames, int total_tiles, int total_chunks, int win_max, int nst,
                   int *err, int check_stop, int passes) {
    assign_pipe_body<false, SAME, MINB, ROWS, TH, true>(frames, n_frames, total_tiles, win_max, nst, err, check_stop,
                                                        passes, total_chunks);
}

// Resident CTAs per SM of one instantiation (the query honours the
// kernel's dynamic shared memory opt-in, so that is raised first).
template <bool L, bool SM, int MINB, int ROWS, int TH = 32>
static int pipe_occupancy_of(size_t smem) {
    int blocks = 0;
    if (cudaFuncSetAttribute(k_assign_pipe<L, SM, MINB, ROWS, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_assign_pipe<L, SM, MINB, ROWS, TH>,
                                                      kThreads / ROWS * (TH / 32), smem) != cudaSuccess)
        return 0;
    return blocks;
}

template <bool SM, int MINB, int ROWS, int TH>
static int multi_occupancy_of(size_t smem) {
    int blocks = 0;
    if (cudaFuncSetAttribute(k_assign_multi<SM, MINB, ROWS, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_assign_multi<SM, MINB, ROWS, TH>,
                                                      kThreads / ROWS * (TH / 32), smem) != cudaSuccess)
        return 0;
    return blocks;
}

int assign_pipe_occupancy(bool same, int win_n, int nst, int rows, int tile_h, bool multi) {
    const size_t sm = assign_pipe_smem_bytes(win_n, false, nst, rows, tile_h, multi);
    if (multi) {
        if (tile_h == 64) return rows == 2 && same ? multi_occupancy_of<true, 2, 2, 64>(sm) : 0;
        if (rows == 2) return same ? multi_occupancy_of<true, 4, 2, 32>(sm) : 0;
        const int o4 = same ? multi_occupancy_of<true, 4, 1, 32>(sm) : multi_occupancy_of<false, 4, 1, 32>(sm);
        const int o3 = same ? multi_occupancy_of<true, 3, 1, 32>(sm) : multi_occupancy_of<false, 3, 1, 32>(sm);
        return o4 >= 4 ? o4 : o3;
    }
    if (tile_h == 64) return rows == 2 && same ? pipe_occupancy_of<false, true, 2, 2, 64>(sm) : 0;
    if (rows == 2) return same ? pipe_occupancy_of<false, true, 4, 2>(sm) : 0;
    // The 4-CTA build (64 registers) where shared memory allows, else the 3-CTA build.
    const int o4 = same ? pipe_occupancy_of<false, true, 4, 1>(sm) : pipe_occupancy_of<false, false, 4, 1>(sm);
    const int o3 = same ? pipe_occupancy_of<false, true, 3, 1>(sm) : pipe_occupancy_of<false, false, 3, 1>(sm);
    return o4 >= 4 ? o4 : o3;
}

template <bool L, bool SM, int MINB, int ROWS, int TH = 32>
static cudaError_t launch_pipe_as(const FrameArgs *d_frames, int n, int total_tiles, int win_max, int nst, int grid,
                                  size_t smem, int *err, int check_stop, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_assign_pipe<L, SM, MINB, ROWS, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_assign_pipe<L, SM, MINB, ROWS, TH><<<grid, kThreads / ROWS * (TH / 32), smem, s>>>(d_frames, n, total_tiles,
                                                                                           win_max, nst, err,
                                                                                           check_stop);
    return cudaGetLastError();
}

cudaError_t launch_assign_pipe(const FrameArgs *d_frames, int n, int total_tiles, int win_max, bool same, bool last,
                               int nst, int rows, int tile_h, int ctas_per_sm, int grid, int *err, int check_stop,
                               cudaStream_t s) {
    if (grid > total_tiles) grid = total_tiles;
    if (grid < 1) grid = 1;
    if (nst < 3) nst = 3;
    if (nst > kMaxStages) nst = kMaxStages;
    if (rows == 2 && !same) return cudaErrorInvalidValue;
    if (tile_h != 32 && (tile_h != 64 || rows != 2)) return cudaErrorInvalidValue;
    const size_t smem = assign_pipe_smem_bytes(win_max, last, nst, rows, tile_h);
    if (tile_h == 64)  // 256 threads at 128 registers: 2 CTAs per SM
        return last ? launch_pipe_as<true, true, 2, 2, 64>(d_frames, n, total_tiles, win_max, nst, grid, smem, err,
                                                           check_stop, s)
                    : launch_pipe_as<false, true, 2, 2, 64>(d_frames, n, total_tiles, win_max, nst, grid, smem, err,
                                                            check_stop, s);
    if (rows == 2)
        return last ? launch_pipe_as<true, true, 4, 2>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s)
                    : launch_pipe_as<false, true, 4, 2>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s);
    const bool wide = ctas_per_sm >= 4;  // 64-register build
    if (same) {
        if (last)
            return wide ? launch_pipe_as<true, true, 4, 1>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s)
                        : launch_pipe_as<true, true, 3, 1>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s);
        return wide ? launch_pipe_as<false, true, 4, 1>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s)
                    : launch_pipe_as<false, true, 3, 1>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s);
    }
    if (last)
        return wide ? launch_pipe_as<true, false, 4, 1>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s)
                    : launch_pipe_as<true, false, 3, 1>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s);
    return wide ? launch_pipe_as<false, false, 4, 1>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s)
                : launch_pipe_as<false, false, 3, 1>(d_frames, n, total_tiles, win_max, nst, grid, smem, err, check_stop, s);
}

// Cooperative launch (every CTA resident at once: the fused kernel's CTAs
// wait on one another's phase counters).
template <bool SM, int MINB, int ROWS, int TH>
static cudaError_t launch_multi_as(const FrameArgs *d_frames, int n, int total_tiles, int total_chunks, int win_max,
                                   int nst, int passes, int grid, size_t smem, int *err, int check_stop,
                                   cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_assign_multi<SM, MINB, ROWS, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)(kThreads / ROWS * (TH / 32)));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_assign_multi<SM, MINB, ROWS, TH>, d_frames, n, total_tiles, total_chunks,
                              win_max, nst, err, check_stop, passes);
}

cudaError_t launch_assign_multi(const FrameArgs *d_frames, int n, int total_tiles, int total_chunks, int win_max,
                                bool same, int passes, int nst, int rows, int tile_h, int ctas_per_sm, int grid,
                                int *err, int check_stop, cudaStream_t s) {
    if (passes < 1) return cudaSuccess;
    if (grid > total_tiles) grid = total_tiles;
    if (grid < 1) grid = 1;
    if (nst < 3) nst = 3;
    if (nst > kMaxStages) nst = kMaxStages;
    if (rows == 2 && !same) return cudaErrorInvalidValue;
    if (tile_h != 32 && (tile_h != 64 || rows != 2)) return cudaErrorInvalidValue;
    const size_t smem = assign_pipe_smem_bytes(win_max, false, nst, rows, tile_h, true);
    if (tile_h == 64)
        return launch_multi_as<true, 2, 2, 64>(d_frames, n, total_tiles, total_chunks, win_max, nst, passes, grid,
                                               smem, err, check_stop, s);
    if (rows == 2)
        return launch_multi_as<true, 4, 2, 32>(d_frames, n, total_tiles, total_chunks, win_max, nst, passes, grid,
                                               smem, err, check_stop, s);
    const bool wide = ctas_per_sm >= 4;  // 64-register build
    if (same)
        return wide ? launch_multi_as<true, 4, 1, 32>(d_frames, n, total_tiles, total_chunks, win_max, nst, passes,
                                                      grid, smem, err, check_stop, s)
                    : launch_multi_as<true, 3, 1, 32>(d_frames, n, total_tiles, total_chunks, win_max, nst, passes,
                                                      grid, smem, err, check_stop, s);
    return wide ? launch_multi_as<false, 4, 1, 32>(d_frames, n, total_tiles, total_chunks, win_max, nst, passes, grid,
                                                   smem, err, check_stop, s)
                : launch_multi_as<false, 3, 1, 32>(d_frames, n, total_tiles, total_chunks, win_max, nst, passes, grid,
                                                   smem, err, check_stop, s);
}

cudaError_t launch_fill_ring(const FrameArgs *d_frames, int n, int max_ring, cudaStream_t s) {
    k_fill_ring<<<dim3((max_ring + 255) / 256, n), 256, 0, s>>>(d_frames, n, max_ring);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Update: centre = member mean; empty centre keeps position and colour.
// ---------------------------------------------------------------------------

__global__ void k_update(long long *acc, const float *centres_in, float *centres_out, int K, float fix_inv,
                         ConvState *cs, float eps, int it) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (conv_stop(cs, eps, K, it)) {
        if (k == 0) cs->done = 1;
        return;
    }
    float move = 0.0f;
    if (k < K)
        move = update_centre(acc + (size_t)k * 6, centres_in + (size_t)k * 6, centres_out + (size_t)k * 6, fix_inv,
                             eps > 0.0f);
    if (cs) conv_record(cs, __all_sync(0xffffffffu, k < K), eps > 0.0f, move, k == 0, it);
}

__global__ void k_update_batch(const FrameArgs *frames, int n, int total, int it) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = g < total;
    // Consecutive centres share a frame: one lookup per warp (its first
    // lane's frame, correct for every lane below the next frame's base),
    // a lane's own search only across a frame boundary.
    const int g0 = __shfl_sync(0xffffffffu, g, 0);
    int f = find_frame<kCentreBase>(frames, n, min(g0, total - 1));
    if (valid && f + 1 < n && g >= frames[f + 1].centre_base) f = find_frame<kCentreBase>(frames, n, g);
    const int f_lane0 = __shfl_sync(0xffffffffu, f, 0);  // (every lane takes part in each warp primitive)
    const bool uniform = __all_sync(0xffffffffu, valid && f == f_lane0);
    const FrameArgs &a = frames[f];
    const int kk = g - a.centre_base;
    float move = 0.0f;
    bool stop = true;
    if (valid) {
        stop = conv_stop(a.cstate, a.conv_eps, a.ns_c * a.ns_r, it);
        if (stop) {
            if (kk == 0) a.cstate->done = 1;
        } else {
            const size_t k = (size_t)kk * 6;
            move = update_centre(a.acc + k, a.centres_out + k, a.centres_out + k, 1.0f / a.fix_scale,
                                 a.conv_eps > 0.0f);
            if (a.ctab) {
                const int r = kk / a.ns_c, c = kk - r * a.ns_c;
                write_ctab(a.ctab + ((size_t)(r + 1) * (a.ns_c + 2) + c + 1) * kCtabRec, a.centres_out + k);
            }
        }
    }
    // (a stopped frame stops for all its centres, so a uniform warp is all
    // stopped or all running)
    if (uniform) {
        if (!stop && a.cstate) conv_record(a.cstate, true, a.conv_eps > 0.0f, move, kk == 0, it);
    } else if (valid && !stop && a.cstate) {
        conv_record(a.cstate, false, a.conv_eps > 0.0f, move, kk == 0, it);
    }
}

// Adds each lane's pixel (fixed-point features, x, y, 1 in v) to the sums
// of its label `key` (< 0: nothing to add), one global atomic per (label,
// component) for all lanes of the warp with that label. Every lane of the
// warp must call it.
__device__ __forceinline__ void add_pixel_sums(long long *acc, int key, const int (&v)[6]) {
    const int lane = threadIdx.x & 31;
    unsigned pending = __ballot_sync(kFull, key >= 0);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int k = __shfl_sync(kFull, key, leader);
        const bool mine = key == k;
        const unsigned grp = __ballot_sync(kFull, mine);
        int s[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) s[c] = __reduce_add_sync(kFull, mine ? v[c] : 0);
        if (lane == leader) {
            unsigned long long *g = reinterpret_cast<unsigned long long *>(acc) + (size_t)k * 6;
#pragma unroll
            for (int c = 0; c < 6; ++c) atomicAdd(&g[c], (unsigned long long)(long long)s[c]);
        }
        pending &= ~grp;
    }
}

// The fixed-point features, coordinates and count of pixel (x, y) when its
// label k lies in [0, K): returns k, else -1.
__device__ __forceinline__ int pixel_sums(const float *feat, int H, int P, const int32_t *labels, int W, int K,
                                          float fs, int x, int y, int (&v)[6]) {
    const int k = labels[(size_t)y * W + x];
    if (k < 0 || k >= K) return -1;
    const size_t plane = (size_t)H * P, off = (size_t)y * P + x;
    v[0] = __float2int_rn(feat[off] * fs);
    v[1] = __float2int_rn(feat[plane + off] * fs);
    v[2] = __float2int_rn(feat[2 * plane + off] * fs);
    v[3] = x;
    v[4] = y;
    v[5] = 1;
    return k;
}

// Sums of the pixels of each label from an explicit label map (an update
// from given labels, e.g. a learned warm start). One thread per pixel;
// warp-aggregated global atomics.
__global__ void k_accumulate_labels(const float *feat, int W, int H, int P, const int32_t *labels, int K,
                                    long long *acc, float fs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        int v[6] = {0, 0, 0, 0, 0, 0};
        const int key = x < W ? pixel_sums(feat, H, P, labels, W, K, fs, x, y, v) : -1;
        add_pixel_sums(acc, key, v);
    }
}

// The same for every frame of a batch that has an initial label map
// (init_labels, e.g. a network's prediction), over the rows of all frames in
// one index space; the first update then takes the member means.
__global__ void __launch_bounds__(128) k_accumulate_labels_batch(const FrameArgs *frames, int n, int total_rows) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    for (int gr = blockIdx.y; gr < total_rows; gr += gridDim.y) {
        const FrameArgs &a = frames[find_frame<kRowBase>(frames, n, gr)];
        if (!a.init_labels) continue;  // (the same for the whole block)
        int v[6] = {0, 0, 0, 0, 0, 0};
        const int key = x < a.W ? pixel_sums(a.feat, a.H, a.P, a.init_labels, a.W, a.ns_c * a.ns_r, a.fix_scale, x,
                                             gr - a.row_base, v)
                                : -1;
        add_pixel_sums(a.acc, key, v);
    }
}

// Stand-alone conversion into planar features with pitch P (2D grid: x
// tiles of 128 pixels, rows strided by gridDim.y).
__global__ void k_convert(ConvConsts cc, const uint8_t *rgb, int W, int H, int C, float *feat, int P) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    const size_t plane = (size_t)H * P;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        const uint8_t *p = rgb + ((size_t)y * W + x) * C;
        float f0, f1, f2;
        convert_pixel(cc, p[0], p[1], p[2], g_lut, f0, f1, f2);
        const size_t off = (size_t)y * P + x;
        feat[off] = f0;
        feat[plane + off] = f1;
        feat[2 * plane + off] = f2;
    }
}

// Batched conversion pre-pass (Sec. 4's colour conversion): RGB -> planar
// features of every frame, 4 pixels per thread; blockIdx.y strides over the
// concatenated rows of all frames. Feature rows have a pitch P that is a
// multiple of 4, so each plane takes one 16-byte store per thread.
__global__ void __launch_bounds__(128) k_convert_batch(const FrameArgs *frames, int n, int total_rows) {
    __shared__ float lut[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = g_lut[i];
    __syncthreads();
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    for (int gr = blockIdx.y; gr < total_rows; gr += gridDim.y) {
        const int f = find_frame<kRowBase>(frames, n, gr);
        const FrameArgs &a = frames[f];
        const int W = a.W, C = a.C;
        if (x0 >= W) continue;
        const int y = gr - a.row_base;
        // Constants in registers: the feature stores below could alias the
        // frame table as far as the compiler knows.
        const ConvConsts cc = a.conv;
        const bool rgb_vec = a.rgb_vec != 0;
        float *const feat = a.feat;
        const size_t plane = (size_t)a.H * a.P, off = (size_t)y * a.P + x0;
        const uint8_t *p = a.rgb + ((size_t)y * W + x0) * C;
        unsigned r[kPPT], g[kPPT], b[kPPT];
        if (rgb_vec && C == 3) {
            const uint32_t *q = reinterpret_cast<const uint32_t *>(p);
            const uint32_t w0 = __ldg(q), w1 = __ldg(q + 1), w2 = __ldg(q + 2);
            r[0] = w0 & 255; g[0] = (w0 >> 8) & 255; b[0] = (w0 >> 16) & 255; r[1] = w0 >> 24;
            g[1] = w1 & 255; b[1] = (w1 >> 8) & 255; r[2] = (w1 >> 16) & 255; g[2] = w1 >> 24;
            b[2] = w2 & 255; r[3] = (w2 >> 8) & 255; g[3] = (w2 >> 16) & 255; b[3] = w2 >> 24;
        } else if (rgb_vec) {
            const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
            const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                r[j] = w[j] & 255; g[j] = (w[j] >> 8) & 255; b[j] = (w[j] >> 16) & 255;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kPPT; ++j) {
                const bool ok = x0 + j < W;
                r[j] = ok ? p[j * C + 0] : 0;
                g[j] = ok ? p[j * C + 1] : 0;
                b[j] = ok ? p[j * C + 2] : 0;
            }
        }
        float f0[kPPT], f1[kPPT], f2[kPPT];
#pragma unroll
        for (int j = 0; j < kPPT; ++j) convert_pixel(cc, r[j], g[j], b[j], lut, f0[j], f1[j], f2[j]);
        *reinterpret_cast<float4 *>(feat + off) = make_float4(f0[0], f0[1], f0[2], f0[3]);
        *reinterpret_cast<float4 *>(feat + plane + off) = make_float4(f1[0], f1[1], f1[2], f1[3]);
        *reinterpret_cast<float4 *>(feat + 2 * plane + off) = make_float4(f2[0], f2[1], f2[2], f2[3]);
    }
}

// ---------------------------------------------------------------------------
// Connectivity: one double-buffered pass, 4 pixels per thread.
// ---------------------------------------------------------------------------

// Majority rule for one pixel: own label and its neighbours in the order
// left, up, right, down, with in-image flags.
__device__ __forceinline__ int32_t connect_rule(int32_t own, const int32_t (&nb)[4], const bool (&ok)[4]) {
    bool any = false, all_differ = true;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        any |= ok[j];
        all_differ &= !ok[j] || nb[j] != own;
    }
    if (!any || !all_differ) return own;
    int32_t result = own;
    int best_count = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!ok[j]) continue;
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) cnt += (ok[q] && nb[q] == nb[j]) ? 1 : 0;
        if (cnt > best_count) {
            best_count = cnt;
            result = nb[j];
        }
    }
    return result;
}

__device__ __forceinline__ void connect_row4(const int32_t *__restrict__ in, int32_t *__restrict__ out, int W, int H,
                                             int x0, int y, bool vec) {
    const size_t row = (size_t)y * W;
    int32_t c[4] = {0, 0, 0, 0}, up[4] = {0, 0, 0, 0}, dn[4] = {0, 0, 0, 0};
    if (vec) {
        const int4 a = __ldg(reinterpret_cast<const int4 *>(in + row + x0));
        c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
        if (y > 0) {
            const int4 u = __ldg(reinterpret_cast<const int4 *>(in + row - W + x0));
            up[0] = u.x; up[1] = u.y; up[2] = u.z; up[3] = u.w;
        }
        if (y < H - 1) {
            const int4 d = __ldg(reinterpret_cast<const int4 *>(in + row + W + x0));
            dn[0] = d.x; dn[1] = d.y; dn[2] = d.z; dn[3] = d.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool okx = x0 + j < W;
            c[j] = okx ? __ldg(in + row + x0 + j) : 0;
            up[j] = (okx && y > 0) ? __ldg(in + row - W + x0 + j) : 0;
            dn[j] = (okx && y < H - 1) ? __ldg(in + row + W + x0 + j) : 0;
        }
    }
    const int32_t left = x0 > 0 ? __ldg(in + row + x0 - 1) : 0;
    const int32_t right = x0 + 4 < W ? __ldg(in + row + x0 + 4) : 0;
    int32_t r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int x = x0 + j;
        const int32_t nb[4] = {j > 0 ? c[j - 1] : left, up[j], j < 3 ? c[j + 1] : right, dn[j]};
        const bool ok[4] = {x > 0, y > 0, x < W - 1, y < H - 1};
        r[j] = connect_rule(c[j], nb, ok);
    }
    if (vec) {
        *reinterpret_cast<int4 *>(out + row + x0) = make_int4(r[0], r[1], r[2], r[3]);
    } else {
        for (int j = 0; j < 4 && x0 + j < W; ++j) out[row + x0 + j] = r[j];
    }
}

__global__ void k_connectivity(const int32_t *__restrict__ in, int32_t *__restrict__ out, int W, int H, int vec) {
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= W) return;
    for (int y = blockIdx.y; y < H; y += gridDim.y) connect_row4(in, out, W, H, x0, y, vec != 0);
}

// pass 0: labels -> lbl_tmp; pass 1: lbl_tmp -> labels. blockIdx.y strides
// over the concatenated rows of all frames.
__global__ void k_connectivity_batch(const FrameArgs *frames, int n, int total_rows, int pass) {
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    for (int gr = blockIdx.y; gr < total_rows; gr += gridDim.y) {
        const int f = find_frame<kRowBase>(frames, n, gr);
        const FrameArgs &a = frames[f];
        if (x0 >= a.W) continue;
        const int32_t *in = pass == 0 ? a.labels : a.lbl_tmp;
        int32_t *out = pass == 0 ? a.lbl_tmp : a.labels;
        connect_row4(in, out, a.W, a.H, x0, gr - a.row_base, a.labels_vec != 0);
    }
}

// Both connectivity passes fused, streaming down vertical strips. A warp
// holds 128 columns [sx - 4, sx + 124) of one strip (lane l: columns
// sx - 4 + 4l .. +3) and walks down a segment of rows with a rolling window
// of input rows and first-pass rows in registers (horizontal neighbours by
// shuffles): input row q + 2 gives the first pass at row q + 1, which gives
// the second pass at row q. Lanes 1..30 write columns [sx, sx + 120); the
// two outer lanes only supply neighbours. Every pixel sees exactly the
// inputs of the two separate passes, so the result equals theirs.
//
// Positions outside the image hold negative sentinels, one per side (left
// -1, above -2, right -3, below -4): a sentinel never equals a label or
// another side's sentinel, which is all the rule needs to skip missing
// neighbours.
namespace {
constexpr int kConnOut = 120;   // output columns per strip
constexpr int kConnSeg = 64;    // output rows per segment

__device__ __forceinline__ int32_t conn_col_sentinel(int x, int W, int32_t v) {
    return x < 0 ? -1 : (x >= W ? -3 : v);
}

__device__ __forceinline__ int4 conn_load_row(const int32_t *in, int W, int H, int y, int x0, bool vec) {
    if (y < 0) return make_int4(-2, -2, -2, -2);
    if (y >= H) return make_int4(-4, -4, -4, -4);
    const int32_t *row = in + (size_t)y * W;
    if (vec && x0 >= 0 && x0 + 3 < W) return __ldg(reinterpret_cast<const int4 *>(row + x0));
    int4 v;
    v.x = (x0 >= 0 && x0 < W) ? __ldg(row + x0) : conn_col_sentinel(x0, W, 0);
    v.y = (x0 + 1 >= 0 && x0 + 1 < W) ? __ldg(row + x0 + 1) : conn_col_sentinel(x0 + 1, W, 0);
    v.z = (x0 + 2 >= 0 && x0 + 2 < W) ? __ldg(row + x0 + 2) : conn_col_sentinel(x0 + 2, W, 0);
    v.w = (x0 + 3 >= 0 && x0 + 3 < W) ? __ldg(row + x0 + 3) : conn_col_sentinel(x0 + 3, W, 0);
    return v;
}

// Sentinels back into a first-pass row (its values outside the image are
// meaningless): the whole row when y is outside, else the lane's columns
// outside (edge lanes only).
__device__ __forceinline__ int4 conn_mask_row(int4 v, int W, int H, int y, int x0, bool edge_lane) {
    if (y < 0) return make_int4(-2, -2, -2, -2);
    if (y >= H) return make_int4(-4, -4, -4, -4);
    if (edge_lane) {
        v.x = conn_col_sentinel(x0, W, v.x);
        v.y = conn_col_sentinel(x0 + 1, W, v.y);
        v.z = conn_col_sentinel(x0 + 2, W, v.z);
        v.w = conn_col_sentinel(x0 + 3, W, v.w);
    }
    return v;
}

// The rule for a pixel none of whose neighbours (left, up, right, down;
// sentinels for missing ones) carries its label: the neighbours' majority,
// the first in that order among the largest counts. With at most four
// values, the left one wins whenever it matches another; else the upper one
// when it matches the right or lower one; else the right one when it matches
// the lower one; else all are distinct and the first valid one wins. No
// valid neighbour at all keeps the label.
__device__ __forceinline__ int32_t conn_majority(int32_t own, int32_t l, int32_t u, int32_t r, int32_t d) {
    const bool el = l == u || l == r || l == d, eu = u == r || u == d, er = r == d;
    const int32_t fv = l >= 0 ? l : (u >= 0 ? u : (r >= 0 ? r : d));
    const int32_t res = el ? l : (eu ? u : (er ? r : fv));
    return res >= 0 ? res : own;
}
// The same where all four neighbours are labels (no sentinel): the first
// valid one is the left one, and the result is always a label.
__device__ __forceinline__ int32_t conn_majority_inner(int32_t l, int32_t u, int32_t r, int32_t d) {
    const bool el = l == u || l == r || l == d, eu = u == r || u == d, er = r == d;
    return el ? l : (eu ? u : (er ? r : l));
}

// One pass of the majority rule at row y for the lane's 4 pixels, from the
// rows above, at and below y (left/right neighbours across lanes). A pixel
// keeps its label when a neighbour shares it (the common case); the
// majority is evaluated only when some pixel of the warp needs it. INNER:
// every neighbour the warp's results depend on is inside the image.
template <bool INNER>
__device__ __forceinline__ int4 conn_rule4(const int4 &up, const int4 &c, const int4 &dn) {
    const int32_t left = __shfl_up_sync(0xffffffffu, c.w, 1), right = __shfl_down_sync(0xffffffffu, c.x, 1);
    const int32_t cc[4] = {c.x, c.y, c.z, c.w}, uu[4] = {up.x, up.y, up.z, up.w}, dd[4] = {dn.x, dn.y, dn.z, dn.w};
    bool need[4];
    bool any_need = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int32_t l = j > 0 ? cc[j - 1] : left, r = j < 3 ? cc[j + 1] : right;
        need[j] = l != cc[j] && uu[j] != cc[j] && r != cc[j] && dd[j] != cc[j];
        any_need |= need[j];
    }
    int32_t res[4] = {cc[0], cc[1], cc[2], cc[3]};
    if (__any_sync(0xffffffffu, any_need)) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int32_t l = j > 0 ? cc[j - 1] : left, r = j < 3 ? cc[j + 1] : right;
            if (need[j]) res[j] = INNER ? conn_majority_inner(l, uu[j], r, dd[j]) : conn_majority(cc[j], l, uu[j], r, dd[j]);
        }
    }
    return make_int4(res[0], res[1], res[2], res[3]);
}
}  // namespace

__global__ void __launch_bounds__(256, 4) k_connectivity2_batch(const FrameArgs *frames, int n, int total_units) {
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (int unit = blockIdx.x * warps + (threadIdx.x >> 5); unit < total_units; unit += gridDim.x * warps) {
        const int f = find_frame<kStripBase>(frames, n, unit);
        const FrameArgs &a = frames[f];
        const int W = a.W, H = a.H;
        const int local = unit - a.strip_base, seg = local / a.strips_x, strip = local - seg * a.strips_x;
        const int sx = strip * kConnOut, x0 = sx - 4 + 4 * lane;
        const int ry0 = seg * kConnSeg, ry1 = min(ry0 + kConnSeg, H);
        const bool vec = (W & 3) == 0;
        const int32_t *in = a.lbl_tmp;
        const bool edge_lane = x0 < 0 || x0 + 3 >= W;
        // Input rows q .. q + 2 (q + 3 in flight) and first-pass rows q - 1, q.
        int4 a_m2 = conn_load_row(in, W, H, ry0 - 2, x0, vec), a_m1 = conn_load_row(in, W, H, ry0 - 1, x0, vec);
        int4 a0 = conn_load_row(in, W, H, ry0, x0, vec), a1 = conn_load_row(in, W, H, ry0 + 1, x0, vec);
        int4 a2 = conn_load_row(in, W, H, ry0 + 2, x0, vec);
        int4 l_m1 = conn_mask_row(conn_rule4<false>(a_m2, a_m1, a0), W, H, ry0 - 1, x0, edge_lane);
        int4 l0 = conn_mask_row(conn_rule4<false>(a_m1, a0, a1), W, H, ry0, x0, edge_lane);
        // Columns sx - 4 .. sx + 123 all inside the image: no lane holds a
        // sentinel column, so rows 1 .. H - 3 take the rule without them.
        const bool inner_cols = sx >= 4 && sx + 124 <= W;
        const bool writer = lane >= 1 && lane <= 30;
        const bool out_vec = vec && a.labels_vec && x0 >= 0 && x0 + 3 < W;
        for (int q = ry0; q < ry1; ++q) {
            const int4 a3 = conn_load_row(in, W, H, q + 3, x0, vec);  // one row ahead of its use
            int4 l1, o;
            if (inner_cols && q >= 1 && q + 2 < H) {
                // input rows q .. q + 2 and first-pass rows q - 1 .. q + 1
                // are all inside the image
                l1 = conn_rule4<true>(a0, a1, a2);
                o = conn_rule4<true>(l_m1, l0, l1);
            } else {
                l1 = conn_mask_row(conn_rule4<false>(a0, a1, a2), W, H, q + 1, x0, edge_lane);
                o = conn_rule4<false>(l_m1, l0, l1);
            }
            if (writer) {
                int32_t *out = a.labels + (size_t)q * W;
                if (out_vec) {
                    *reinterpret_cast<int4 *>(out + x0) = o;
                } else {
                    const int32_t ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (x0 + j >= 0 && x0 + j < W) out[x0 + j] = ov[j];
                }
            }
            l_m1 = l0;
            l0 = l1;
            a0 = a1;
            a1 = a2;
            a2 = a3;
        }
    }
}

// ---------------------------------------------------------------------------
// Component-based connectivity (the original SLIC's notion of enforcing
// connectivity, Sec. 2), an alternative to the paper's local rule: the
// 4-connected segments of equal labels, in scan order of their first pixel;
// a segment of at most min_size pixels joins the segment of its first
// pixel's left neighbour (its upper one in column 0), the segment of pixel 0
// is kept, and kept segments are numbered 0, 1, ... in scan order.
//
// Union-find over pixel indices: a pixel's parent always has a smaller
// index, so each component's root is its first pixel in scan order. The
// pixels of all frames of a call form one index space (frame f holds base_f
// .. base_f + W_f*H_f - 1). Stages:
//   1. per 32x32 tile, union-find in shared memory; every pixel's parent is
//      its tile-local root (the component's first pixel within the tile),
//      which carries its size within the tile and goes into a list;
//   2. unions across the tile edges (global memory), only for edge pixels;
//   3. per tile-local root only: its component's root and the sizes;
//   4-5. per component root only: keep it or join a neighbour's segment,
//      then follow the joins to a kept root; kept roots are marked in a
//      bitmap;
//   6. ranks of the kept roots (a scan of the bitmap's population counts);
//   7. per tile-local root: its segment's new label; then per pixel: the
//      label of its tile-local root.
// Every walk is bounded; a walk that gives up sets bit 1 of *err, and the
// indices it leaves behind stay in range.
// ---------------------------------------------------------------------------
namespace {
constexpr unsigned kCclSteps = 1u << 22;
constexpr int kCclTile = 32;                          // tile side (pixels)
constexpr int kCclThreads = 128;                      // per tile: 8 pixels per thread
constexpr int kScanThreads = 256, kScanPer = 8, kScanBlock = kScanThreads * kScanPer;
}  // namespace

// Step limit of every walk below (kCclSteps; lowered only by fault
// injection, to make walks give up in tests of the timeout reporting).
__device__ unsigned g_ccl_steps = kCclSteps;

namespace {
__device__ __forceinline__ int ccl_find(const int *parent, int i, int *err) {
    const unsigned lim = g_ccl_steps;
    for (unsigned n = 0; n < lim; ++n) {
        const int p = __ldcg(parent + i);
        if (p == i) return i;
        i = p;
    }
    atomicOr(err, 2);
    return i;
}

// Link the trees of a and b: the larger root takes the smaller as parent
// (atomicMin; a root changed meanwhile is followed and the link retried).
__device__ __forceinline__ void ccl_union(int *parent, int a, int b, int *err) {
    const unsigned lim = g_ccl_steps;
    for (unsigned n = 0; n < lim; ++n) {
        a = ccl_find(parent, a, err);
        b = ccl_find(parent, b, err);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(parent + a, b);
        if (old == a) return;
        a = old;
    }
    atomicOr(err, 2);
}

// The same two operations on a tile's parents in shared memory.
// (with path halving: an entry on the way is pointed at its grandparent,
// an ancestor, which concurrent walks and links tolerate)
__device__ __forceinline__ int ccl_find_s(int *par, int i, int *err) {
    volatile int *vp = par;
    const unsigned lim = g_ccl_steps;
    for (unsigned n = 0; n < lim; ++n) {
        const int p = vp[i];
        if (p == i) return i;
        const int gp = vp[p];
        if (gp != p) vp[i] = gp;
        i = gp;
    }
    atomicOr(err, 2);
    return i;
}
__device__ __forceinline__ void ccl_union_s(int *par, int a, int b, int *err) {
    const unsigned lim = g_ccl_steps;
    for (unsigned n = 0; n < lim; ++n) {
        a = ccl_find_s(par, a, err);
        b = ccl_find_s(par, b, err);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(par + a, b);
        if (old == a) return;
        a = old;
    }
    atomicOr(err, 2);
}
}  // namespace

// The frames of a call: one travels in the launch itself, several in a
// device table.
struct CclFrames {
    const CclFrame *table;
    CclFrame one;
    int n;
};

// The frame holding global pixel g (last base <= g), or tile t (last tile
// base <= t).
__device__ __forceinline__ CclFrame ccl_frame_of(const CclFrames &fr, int g) {
    if (fr.n == 1) return fr.one;
    int lo = 0, hi = fr.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fr.table[mid].base <= g) lo = mid;
        else hi = mid - 1;
    }
    return fr.table[lo];
}
__device__ __forceinline__ CclFrame ccl_frame_of_tile(const CclFrames &fr, int t) {
    if (fr.n == 1) return fr.one;
    int lo = 0, hi = fr.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fr.table[mid].tile_base <= t) lo = mid;
        else hi = mid - 1;
    }
    return fr.table[lo];
}

// Stage 1: a CTA per 32x32 tile, a warp per tile row at a time. Parents in
// shared memory (tile-local indices in row-major order, which is scan order
// within the tile): each pixel starts at the first pixel of its horizontal
// run (a ballot over the row), vertical links join runs (a pixel whose left
// neighbour makes the same vertical link needs none), then every pixel is
// compressed to its tile-local root. Output: every pixel's global parent is
// its tile-local root; a tile-local root's count is its size within the
// tile, and it is appended to the list lroots[0 .. *n_lroots).
__global__ void __launch_bounds__(kCclThreads) k_ccl_local(CclFrames fr, int *parent, int *count, int *lroots,
                                                            int *n_lroots, int *err) {
    __shared__ int32_t lab[kCclTile * kCclTile];
    __shared__ int par[kCclTile * kCclTile];
    __shared__ int cnt[kCclTile * kCclTile];
    const CclFrame f = ccl_frame_of_tile(fr, blockIdx.x);
    const int local = blockIdx.x - f.tile_base, tiles_x = (f.W + kCclTile - 1) / kCclTile;
    const int ty = local / tiles_x, tx = local - ty * tiles_x;
    const int x0 = tx * kCclTile, y0 = ty * kCclTile;
    const int tw = min(kCclTile, f.W - x0), th = min(kCclTile, f.H - y0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kRowsPerPass = kCclThreads / 32;
    const bool col_ok = lane < tw;
    for (int ly = warp; ly < kCclTile; ly += kRowsPerPass) {
        const int i = ly * kCclTile + lane;
        const bool ok = col_ok && ly < th;
        const int32_t v = ok ? f.in[(size_t)(y0 + ly) * f.W + x0 + lane] : 0;
        lab[i] = v;
        cnt[i] = 0;
        const int32_t left = __shfl_up_sync(kFull, v, 1);
        const bool start = lane == 0 || left != v;
        const unsigned starts = __ballot_sync(kFull, start) & (kFull >> (31 - lane));
        par[i] = ly * kCclTile + (31 - __clz(starts));
    }
    __syncthreads();
    for (int ly = warp + (warp == 0 ? kRowsPerPass : 0); ly < th; ly += kRowsPerPass) {
        if (!col_ok) continue;
        const int i = ly * kCclTile + lane;
        const int32_t v = lab[i];
        if (lab[i - kCclTile] != v) continue;
        if (lane > 0 && lab[i - 1] == v && lab[i - kCclTile - 1] == v) continue;
        ccl_union_s(par, i, i - kCclTile, err);
    }
    __syncthreads();
    // Roots are always run starts (a link goes from a root to a root), so
    // only the starts need a walk: each adds its run's length to its root's
    // size, and the run's pixels take its root (no parent points at a pixel
    // that is not a run start, so those entries can change freely).
    for (int ly = warp; ly < th; ly += kRowsPerPass) {
        const int i = ly * kCclTile + lane;
        const int32_t v = lab[i];
        const bool start = col_ok && (lane == 0 || lab[i - 1] != v);
        const unsigned st = __ballot_sync(kFull, start);
        int r = i;
        if (start) {
            r = ccl_find_s(par, i, err);
            const unsigned after = st & ~(kFull >> (31 - lane));
            atomicAdd(&cnt[r], (after ? __ffs(after) - 1 : tw) - lane);
        }
        r = __shfl_sync(kFull, r, 31 - __clz(st & (kFull >> (31 - lane))));
        if (col_ok) par[i] = r;
    }
    __syncthreads();
    // Parents out; the tile's roots go into the list with one global atomic
    // per tile (a slot range), ordered by warp and row within it.
    __shared__ int wbase[kRowsPerPass + 1];
    int mine = 0;
    for (int ly = warp; ly < th; ly += kRowsPerPass) {
        const int i = ly * kCclTile + lane;
        const int r = par[i];
        const int g = f.base + (y0 + ly) * f.W + x0 + lane;
        if (col_ok) parent[g] = f.base + (y0 + r / kCclTile) * f.W + x0 + (r & (kCclTile - 1));
        const bool is_root = col_ok && r == i;
        if (is_root) count[g] = cnt[i];
        mine += __popc(__ballot_sync(kFull, is_root));
    }
    if (lane == 0) wbase[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < kRowsPerPass; ++w) {
            const int c = wbase[w];
            wbase[w] = run;
            run += c;
        }
        wbase[kRowsPerPass] = run ? atomicAdd(n_lroots, run) : 0;
    }
    __syncthreads();
    int slot = wbase[kRowsPerPass] + wbase[warp];
    for (int ly = warp; ly < th; ly += kRowsPerPass) {
        const int i = ly * kCclTile + lane;
        const bool is_root = col_ok && par[i] == i;
        const unsigned roots = __ballot_sync(kFull, is_root);
        if (is_root) lroots[slot + __popc(roots & ((1u << lane) - 1))] = f.base + (y0 + ly) * f.W + x0 + lane;
        slot += __popc(roots);
    }
}

// Stage 2: unions across the tile's left and upper edges (a thread per edge
// pixel). A pair whose neighbours along the edge are an equal-labelled pair
// is skipped: both sides are connected inside their tiles.
__global__ void __launch_bounds__(2 * kCclTile) k_ccl_border(CclFrames fr, int *parent, int *err) {
    const CclFrame f = ccl_frame_of_tile(fr, blockIdx.x);
    const int local = blockIdx.x - f.tile_base, tiles_x = (f.W + kCclTile - 1) / kCclTile;
    const int ty = local / tiles_x, tx = local - ty * tiles_x;
    const int x0 = tx * kCclTile, y0 = ty * kCclTile, W = f.W;
    const int tw = min(kCclTile, W - x0), th = min(kCclTile, f.H - y0);
    const int t = threadIdx.x & (kCclTile - 1);
    if (threadIdx.x < kCclTile) {  // left edge: (x0, y0 + t) with (x0 - 1, y0 + t)
        if (x0 == 0 || t >= th) return;
        const int i = (y0 + t) * W + x0;
        const int32_t v = f.in[i];
        if (f.in[i - 1] != v) return;
        if (t > 0 && f.in[i - W] == v && f.in[i - W - 1] == v) return;
        ccl_union(parent, f.base + i, f.base + i - 1, err);
    } else {  // upper edge: (x0 + t, y0) with (x0 + t, y0 - 1)
        if (y0 == 0 || t >= tw) return;
        const int i = y0 * W + x0 + t;
        const int32_t v = f.in[i];
        if (f.in[i - W] != v) return;
        if (t > 0 && f.in[i - 1] == v && f.in[i - W - 1] == v) return;
        ccl_union(parent, f.base + i, f.base + i - W, err);
    }
}

// Stage 3, per tile-local root L: its component's root R (the parent of L
// becomes R), and L's size added into R's. R's own entry is only added into
// (R is a tile-local root that finds itself), so the sums need no order.
__global__ void k_ccl_roots(int G, const int *lroots, const int *n_lroots, int *parent, int *count, int *err) {
    const int nr = *n_lroots;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += gridDim.x * blockDim.x) {
        const int L = lroots[k];
        int R = ccl_find(parent, L, err);
        if ((unsigned)R >= (unsigned)G) R = L;  // (only after a walk gave up)
        if (R != L) {
            parent[L] = R;
            atomicAdd(count + R, __ldcg(count + L));
        }
    }
}

// Stage 4, per component root R (a tile-local root that is its own parent):
// itself when kept (marked in the bitmap of kept roots), else the root of
// its first pixel's left (or, in column 0, upper) neighbour, two steps away
// (pixel -> tile-local root -> root); a frame's first pixel is always kept.
__global__ void k_ccl_decide(CclFrames fr, const int *lroots, const int *n_lroots, const int *parent,
                             const int *count, int *target, unsigned *kept) {
    const int nr = *n_lroots;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += gridDim.x * blockDim.x) {
        const int g = lroots[k];
        if (parent[g] != g) continue;
        const CclFrame f = ccl_frame_of(fr, g);
        const int i = g - f.base;
        int t = g;
        if (i != 0 && count[g] <= f.min_size) t = parent[parent[i % f.W > 0 ? g - 1 : g - f.W]];
        target[g] = t;
        if (t == g) atomicOr(kept + (g >> 5), 1u << (g & 31));
    }
}

// Stage 5, per component root: follow the joins to the kept segment (chains
// point to smaller indices and end at a kept root; in place, every value
// written stays on the chain). Every step is checked to stay in [0, G).
__global__ void k_ccl_resolve(int G, const int *lroots, const int *n_lroots, const int *parent, int *target,
                              int *err) {
    const int nr = *n_lroots;
    const unsigned lim = g_ccl_steps;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += gridDim.x * blockDim.x) {
        const int g = lroots[k];
        if (parent[g] != g) continue;
        int t = target[g];
        unsigned n = 0;
        for (; n < lim; ++n) {
            if ((unsigned)t >= (unsigned)G) {
                t = g;
                n = lim;
                break;
            }
            const int u = __ldcg(target + t);
            if (u == t) break;
            t = u;
        }
        if (n == lim) atomicOr(err, 2);
        target[g] = t;
    }
}

// Stage 6a: exclusive scan of the kept bitmap's population counts, block by
// block (kScanBlock words): rank[w] within the block, totals[block].
__global__ void __launch_bounds__(kScanThreads) k_ccl_scan_block(int nw, const unsigned *kept, int *rank,
                                                                  int *totals) {
    __shared__ int warp_sum[kScanThreads / 32];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int f[kScanPer], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        const int w = base + j;
        f[j] = w < nw ? __popc(kept[w]) : 0;
        sum += f[j];
    }
    int incl = sum;  // inclusive scan of the thread sums within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += warp_sum[w];
    int run = before + incl - sum;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        const int w = base + j;
        if (w < nw) rank[w] = run;
        run += f[j];
    }
    if (threadIdx.x == kScanThreads - 1) totals[blockIdx.x] = run;
}

// Exclusive scan of the block totals, in place (one block).
__global__ void __launch_bounds__(1024) k_ccl_scan_totals(int nb, int *totals) {
    __shared__ int warp_sum[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += 1024) {
        const int i = c0 + threadIdx.x;
        const int v = i < nb ? totals[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        int before = carry;
        for (int w = 0; w < warp; ++w) before += warp_sum[w];
        if (i < nb) totals[i] = before + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + incl;
        __syncthreads();
    }
}

namespace {
// Number of kept roots before global index k.
__device__ __forceinline__ int ccl_rank(const unsigned *kept, const int *rank, const int *totals, int k) {
    const int w = k >> 5;
    return rank[w] + totals[w / kScanBlock] + __popc(kept[w] & ((1u << (k & 31)) - 1u));
}
}  // namespace

// Stage 7a, per tile-local root L: the new label of L's segment, the rank of
// its kept root among all kept roots less the rank of the frame's first
// pixel (a kept root, the frame's label 0), into count[L] (sizes are no
// longer needed).
__global__ void k_ccl_final(CclFrames fr, int G, const int *lroots, const int *n_lroots, const int *parent,
                            const int *target, const unsigned *kept, const int *rank, const int *totals, int *count) {
    const int nr = *n_lroots;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += gridDim.x * blockDim.x) {
        const int L = lroots[k];
        const CclFrame f = ccl_frame_of(fr, L);
        int R = parent[L];
        // (out of range only after a walk gave up, which set the error flag:
        // the label is then wrong, the accesses still in bounds)
        if ((unsigned)R >= (unsigned)G) R = L;
        int t = target[R];
        if ((unsigned)t >= (unsigned)G) t = f.base;
        count[L] = ccl_rank(kept, rank, totals, t) - ccl_rank(kept, rank, totals, f.base);
    }
}

// Stage 7b, a CTA per tile: every pixel takes the label of its parent -- its
// tile-local root, or for a tile-local root its segment's root, itself a
// tile-local root of the same segment.
__global__ void __launch_bounds__(kCclThreads) k_ccl_relabel(CclFrames fr, int G, const int *parent,
                                                              const int *labels_of) {
    const CclFrame f = ccl_frame_of_tile(fr, blockIdx.x);
    const int local = blockIdx.x - f.tile_base, tiles_x = (f.W + kCclTile - 1) / kCclTile;
    const int ty = local / tiles_x, tx = local - ty * tiles_x;
    const int x0 = tx * kCclTile, y0 = ty * kCclTile;
    const int tw = min(kCclTile, f.W - x0), th = min(kCclTile, f.H - y0);
    for (int i = threadIdx.x; i < kCclTile * kCclTile; i += kCclThreads) {
        const int lx = i & (kCclTile - 1), ly = i / kCclTile;
        if (lx >= tw || ly >= th) continue;
        const int p = (y0 + ly) * f.W + x0 + lx;
        int L = parent[f.base + p];
        if ((unsigned)L >= (unsigned)G) L = f.base;  // (only after a walk gave up)
        f.out[p] = labels_of[L];
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------

cudaError_t upload_lut(const float *lut256) { return cudaMemcpyToSymbol(g_lut, lut256, 256 * sizeof(float)); }

cudaError_t set_fault_words(unsigned ccl_steps, int abort_copies) {
    cudaError_t e = cudaMemcpyToSymbol(g_ccl_steps, &ccl_steps, sizeof ccl_steps);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_abort_copies, &abort_copies, sizeof abort_copies);
    return e;
}

unsigned ccl_default_steps() { return kCclSteps; }

template <bool F, bool L, bool SM>
static cudaError_t set_smem(int bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_assign<F, L, SM>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_assign_batch<F, L, SM>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t configure_kernels(size_t max_smem) {
    const int b = (int)max_smem;
    cudaError_t e;
    if ((e = set_smem<true, true, true>(b)) != cudaSuccess) return e;
    if ((e = set_smem<true, false, true>(b)) != cudaSuccess) return e;
    if ((e = set_smem<false, true, true>(b)) != cudaSuccess) return e;
    if ((e = set_smem<false, false, true>(b)) != cudaSuccess) return e;
    if ((e = set_smem<true, true, false>(b)) != cudaSuccess) return e;
    if ((e = set_smem<true, false, false>(b)) != cudaSuccess) return e;
    if ((e = set_smem<false, true, false>(b)) != cudaSuccess) return e;
    return set_smem<false, false, false>(b);
}

cudaError_t launch_init_from_rgb(const FrameArgs &a, cudaStream_t s) {
    const int K = a.ns_c * a.ns_r;
    k_init_rgb<<<(K + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_convert_batch(const FrameArgs *d_frames, int n, int total_rows, int max_w, cudaStream_t s) {
    const int threads = 128;
    const dim3 grid((unsigned)((max_w + 4 * threads - 1) / (4 * threads)), (unsigned)std::min(total_rows, 4096));
    k_convert_batch<<<grid, threads, 0, s>>>(d_frames, n, total_rows);
    return cudaGetLastError();
}

int connectivity2_units(int W, int H, int *strips_x) {
    *strips_x = (W + kConnOut - 1) / kConnOut;
    return *strips_x * ((H + kConnSeg - 1) / kConnSeg);
}

cudaError_t launch_connectivity2_batch(const FrameArgs *d_frames, int n, int total_units, int grid, cudaStream_t s) {
    const int per_block = 8;  // warps per 256-thread block, one unit each
    const int need = (total_units + per_block - 1) / per_block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_connectivity2_batch<<<grid, 32 * per_block, 0, s>>>(d_frames, n, total_units);
    return cudaGetLastError();
}

cudaError_t launch_init_batch(const FrameArgs *d_frames, int n, int total_centres, cudaStream_t s) {
    k_init_batch<<<(total_centres + 127) / 128, 128, 0, s>>>(d_frames, n, total_centres);
    return cudaGetLastError();
}

cudaError_t launch_init_from_feat(const float *feat, int W, int H, int P, int S, int ns_c, int ns_r, int perturb,
                                  float *centres, cudaStream_t s) {
    const int K = ns_c * ns_r;
    k_init_feat<<<(K + 127) / 128, 128, 0, s>>>(feat, W, H, P, S, ns_c, ns_r, perturb, centres);
    return cudaGetLastError();
}

cudaError_t launch_zero_acc(long long *acc, int K, cudaStream_t s) {
    const int n = K * 6;
    k_zero_acc<<<(n + 255) / 256, 256, 0, s>>>(acc, n);
    return cudaGetLastError();
}

cudaError_t launch_assign(const FrameArgs &a, bool first, bool last, bool store_feat, size_t smem, cudaStream_t s) {
    const dim3 grid((a.W + kTileW - 1) / kTileW, (a.H + kTileH - 1) / kTileH);
    const int sf = store_feat ? 1 : 0;
    if ((a.S % kPPT) == 0) {
        if (first && last) k_assign<true, true, true><<<grid, kThreads, smem, s>>>(a, sf);
        else if (first) k_assign<true, false, true><<<grid, kThreads, smem, s>>>(a, sf);
        else if (last) k_assign<false, true, true><<<grid, kThreads, smem, s>>>(a, sf);
        else k_assign<false, false, true><<<grid, kThreads, smem, s>>>(a, sf);
    } else {
        if (first && last) k_assign<true, true, false><<<grid, kThreads, smem, s>>>(a, sf);
        else if (first) k_assign<true, false, false><<<grid, kThreads, smem, s>>>(a, sf);
        else if (last) k_assign<false, true, false><<<grid, kThreads, smem, s>>>(a, sf);
        else k_assign<false, false, false><<<grid, kThreads, smem, s>>>(a, sf);
    }
    return cudaGetLastError();
}

cudaError_t launch_assign_batch(const FrameArgs *d_frames, int n, int total_tiles, int win_max, bool same, bool first,
                                bool last, size_t smem, int grid, cudaStream_t s) {
    if (grid > total_tiles) grid = total_tiles;
    if (grid < 1) grid = 1;
    const int N = n, T = total_tiles, Wm = win_max;
    if (same) {
        if (first && last) k_assign_batch<true, true, true><<<grid, kThreads, smem, s>>>(d_frames, N, T, Wm);
        else if (first) k_assign_batch<true, false, true><<<grid, kThreads, smem, s>>>(d_frames, N, T, Wm);
        else if (last) k_assign_batch<false, true, true><<<grid, kThreads, smem, s>>>(d_frames, N, T, Wm);
        else k_assign_batch<false, false, true><<<grid, kThreads, smem, s>>>(d_frames, N, T, Wm);
    } else {
        if (first && last) k_assign_batch<true, true, false><<<grid, kThreads, smem, s>>>(d_frames, N, T, Wm);
        else if (first) k_assign_batch<true, false, false><<<grid, kThreads, smem, s>>>(d_frames, N, T, Wm);
        else if (last) k_assign_batch<false, true, false><<<grid, kThreads, smem, s>>>(d_frames, N, T, Wm);
        else k_assign_batch<false, false, false><<<grid, kThreads, smem, s>>>(d_frames, N, T, Wm);
    }
    return cudaGetLastError();
}

template <bool F, bool L, bool SM>
static int occupancy_of(size_t smem) {
    int blocks = 0;
    if (cudaFuncSetAttribute(k_assign_batch<F, L, SM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_assign_batch<F, L, SM>, kThreads, smem) !=
            cudaSuccess)
        return 0;
    return blocks;
}

int assign_batch_occupancy(bool same, size_t smem) {
    // The four pass kinds share the same shape; take the smallest.
    int b = same ? occupancy_of<false, false, true>(smem) : occupancy_of<false, false, false>(smem);
    const int b2 = same ? occupancy_of<true, false, true>(smem) : occupancy_of<true, false, false>(smem);
    return b2 < b ? b2 : b;
}

cudaError_t launch_update(long long *acc, const float *centres_in, float *centres_out, int K, float fix_inv,
                          ConvState *cstate, float eps, int it, cudaStream_t s) {
    k_update<<<(K + 127) / 128, 128, 0, s>>>(acc, centres_in, centres_out, K, fix_inv, cstate, eps, it);
    return cudaGetLastError();
}

cudaError_t launch_update_batch(const FrameArgs *d_frames, int n, int total_centres, int it, cudaStream_t s) {
    k_update_batch<<<(total_centres + 127) / 128, 128, 0, s>>>(d_frames, n, total_centres, it);
    return cudaGetLastError();
}

static dim3 rows_grid(int W, int H, int bx, int ppt) {
    return dim3((W + bx * ppt - 1) / (bx * ppt), H < 65535 ? H : 65535);
}

cudaError_t launch_accumulate_labels(const float *feat, int W, int H, int P, const int32_t *labels, int K,
                                     long long *acc, float fix_scale, cudaStream_t s) {
    k_accumulate_labels<<<rows_grid(W, H, 128, 1), 128, 0, s>>>(feat, W, H, P, labels, K, acc, fix_scale);
    return cudaGetLastError();
}

cudaError_t launch_accumulate_labels_batch(const FrameArgs *d_frames, int n, int total_rows, int max_w,
                                           cudaStream_t s) {
    const dim3 grid((unsigned)((max_w + 127) / 128), (unsigned)std::min(total_rows, 8192));
    k_accumulate_labels_batch<<<grid, 128, 0, s>>>(d_frames, n, total_rows);
    return cudaGetLastError();
}

cudaError_t launch_convert(const ConvConsts &cc, const uint8_t *rgb, int W, int H, int C, float *feat, int P,
                           cudaStream_t s) {
    k_convert<<<rows_grid(W, H, 128, 1), 128, 0, s>>>(cc, rgb, W, H, C, feat, P);
    return cudaGetLastError();
}

cudaError_t launch_connectivity(const int32_t *in, int32_t *out, int W, int H, cudaStream_t s) {
    const int vec = ((W & 3) == 0 && ((uintptr_t)in & 15) == 0 && ((uintptr_t)out & 15) == 0) ? 1 : 0;
    k_connectivity<<<rows_grid(W, H, 64, 4), 64, 0, s>>>(in, out, W, H, vec);
    return cudaGetLastError();
}

// Scratch of launch_connectivity_components over N pixels: parents, sizes,
// join targets and the list of tile-local roots (N ints each), the kept-root bitmap and
// its ranks (one int per 32 pixels each), the block totals, the root count.
size_t ccl_scratch_ints(long long N) {
    const long long nw = (N + 31) / 32;
    return (size_t)N * 4 + (size_t)nw * 2 + (size_t)((nw + kScanBlock - 1) / kScanBlock) + 64;
}

int ccl_tiles(int W, int H) { return ((W + kCclTile - 1) / kCclTile) * ((H + kCclTile - 1) / kCclTile); }

cudaError_t launch_connectivity_components(const CclFrame *d_table, const CclFrame &one, int n, int G, int tiles,
                                           int *scratch, int *err, cudaStream_t s) {
    CclFrames fr;
    fr.table = d_table;
    fr.one = one;
    fr.n = n;
    const int nw = (G + 31) / 32, nb = (nw + kScanBlock - 1) / kScanBlock, g = (G + 255) / 256;
    int *parent = scratch, *count = scratch + G, *target = scratch + 2 * (size_t)G, *lroots = scratch + 3 * (size_t)G;
    unsigned *kept = reinterpret_cast<unsigned *>(scratch + 4 * (size_t)G);
    int *rank = scratch + 4 * (size_t)G + nw, *totals = rank + nw, *n_lroots = totals + nb;
    cudaError_t e = cudaMemsetAsync(kept, 0, sizeof(unsigned) * (size_t)nw, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_lroots, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    // the root stages run over the root list with a grid sized for the device
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid_roots = std::max(1, std::min(sms * 8, g));
    k_ccl_local<<<tiles, kCclThreads, 0, s>>>(fr, parent, count, lroots, n_lroots, err);
    k_ccl_border<<<tiles, 2 * kCclTile, 0, s>>>(fr, parent, err);
    k_ccl_roots<<<grid_roots, 256, 0, s>>>(G, lroots, n_lroots, parent, count, err);
    k_ccl_decide<<<grid_roots, 256, 0, s>>>(fr, lroots, n_lroots, parent, count, target, kept);
    k_ccl_resolve<<<grid_roots, 256, 0, s>>>(G, lroots, n_lroots, parent, target, err);
    k_ccl_scan_block<<<nb, kScanThreads, 0, s>>>(nw, kept, rank, totals);
    k_ccl_scan_totals<<<1, 1024, 0, s>>>(nb, totals);
    k_ccl_final<<<grid_roots, 256, 0, s>>>(fr, G, lroots, n_lroots, parent, target, kept, rank, totals, count);
    k_ccl_relabel<<<tiles, kCclThreads, 0, s>>>(fr, G, parent, count);
    return cudaGetLastError();
}

cudaError_t launch_connectivity_components(const int32_t *in, int32_t *out, int W, int H, int min_size,
                                           int *scratch, int *err, cudaStream_t s) {
    CclFrame one{in, out, W, min_size, 0, H, 0};
    return launch_connectivity_components(nullptr, one, 1, W * H, ccl_tiles(W, H), scratch, err, s);
}

cudaError_t launch_connectivity_batch(const FrameArgs *d_frames, int n, int total_rows, int max_w, int pass,
                                      cudaStream_t s) {
    k_connectivity_batch<<<rows_grid(max_w, total_rows, 64, 4), 64, 0, s>>>(d_frames, n, total_rows, pass);
    return cudaGetLastError();
}

}  // namespace slicgb
