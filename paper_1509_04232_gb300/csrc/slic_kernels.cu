// SLIC kernels for sm_103a (gSLICr, arXiv 1509.04232, Sec. 3).
//
//   k_init_rgb / k_init_feat  "Cluster center initialisation": one thread per
//                             centre, position = midpoint of the in-image part
//                             of its grid cell, colour = the pixel under it.
//   k_assign<FIRST,LAST>      "Finding the cluster associations" (Eq. 1) for a
//                             32x32-pixel tile, with the tile's window of
//                             centres staged in shared memory. FIRST fuses
//                             "Image space conversion" (RGB bytes in, features
//                             stored once); !LAST fuses the first half of
//                             "Updating the cluster center": per-tile sums of
//                             the members of each window centre, reduced with
//                             warp-wide integer reductions and flushed with
//                             one atomic per (centre, component) per tile.
//   k_update                  second half of the update: centre = sum/count
//                             (empty centre keeps its position and colour).
//   k_connectivity            one pass of "Enforce connectivity".
//
// The sums are exact integers (features in fixed point with a 2^-16
// quantum), so the result is independent of the order in which tiles, warps
// or frames contribute.
#include "slic_internal.cuh"

#include <cstdint>

namespace slicgb {

__device__ float g_lut[256];  // sRGB byte -> linear, filled by the host

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float fsqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float lab_f(const ConvConsts &cc, float t) {
    return t > cc.eps ? cbrtf(t) : fmaf(cc.k_slope, t, cc.k_offset);
}

// Sec. 3 "Image space conversion" for one pixel. `lut` is the sRGB
// linearisation table (shared or global memory).
__device__ __forceinline__ void convert_pixel(const ConvConsts &cc, unsigned r, unsigned g, unsigned b,
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

__global__ void k_init_rgb(FrameArgs a, float *centres, long long *acc) {
    const int K = a.ns_c * a.ns_r;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    float xk, yk;
    int px, py;
    init_centre_position(k, a.W, a.H, a.S, a.ns_c, xk, yk, px, py);
    const uint8_t *p = a.rgb + ((size_t)py * a.W + px) * a.C;
    float f0, f1, f2;
    convert_pixel(a.conv, p[0], p[1], p[2], g_lut, f0, f1, f2);
    float *ck = centres + (size_t)k * 6;
    ck[0] = f0;
    ck[1] = f1;
    ck[2] = f2;
    ck[3] = xk;
    ck[4] = yk;
    ck[5] = 0.0f;
    long long *ak = acc + (size_t)k * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) ak[c] = 0;
}

__global__ void k_init_feat(const float *feat, int W, int H, int P, int S, int ns_c, int ns_r, float *centres) {
    const int K = ns_c * ns_r;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    float xk, yk;
    int px, py;
    init_centre_position(k, W, H, S, ns_c, xk, yk, px, py);
    const size_t plane = (size_t)H * P, off = (size_t)py * P + px;
    float *ck = centres + (size_t)k * 6;
    ck[0] = feat[off];
    ck[1] = feat[plane + off];
    ck[2] = feat[2 * plane + off];
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
// CTA = 32x32-pixel tile, 8 warps; warp w covers the 16x8 block at
// (16*(w%2), 8*(w/2)) of the tile; lane l covers 4 horizontally adjacent
// pixels at (4*(l%4), l/4) of that block, so a warp reads 8 rows of 64
// contiguous bytes per feature plane.
//
// Partial sums for the update: each lane merges runs of equal labels among
// its 4 pixels, each warp reduces equal keys with redux.sync into private
// int32 accumulators in shared memory (a warp covers 128 pixels, so a sum
// is below 128 * 255 * 2^16 < 2^31), and the CTA adds its 8 warps' totals
// in int64 and issues one global atomic per non-zero (centre, component).
// Windows too large for private accumulators (S <= 2) use warp-aggregated
// global atomics instead.

namespace {
constexpr int kWarps = kThreads / 32;
constexpr float kSentinel = 1e18f;
constexpr size_t kPrivateAccLimit = 64 * 1024;
}  // namespace

// Window of cells a tile can reference: the cells its pixels fall in plus
// one ring, clamped to what the grid can offer.
int assign_max_window(int S, int ns_c, int ns_r) {
    const int span = (kTileW - 1) / S + 2;  // cells a 32-px run can touch, misaligned
    const int spanh = (kTileH - 1) / S + 2;
    const int wx = (span < ns_c ? span : ns_c) + 2;
    const int wy = (spanh < ns_r ? spanh : ns_r) + 2;
    return wx * wy;
}

bool assign_direct_acc(int win_n) { return (size_t)kWarps * win_n * 4 * sizeof(int) > kPrivateAccLimit; }

size_t assign_smem_bytes(int win_n, bool first) {
    size_t b = ((size_t)win_n * 20 + 15) & ~(size_t)15;
    if (!assign_direct_acc(win_n)) b += (size_t)kWarps * win_n * 4 * sizeof(int);
    if (first) b += 256 * sizeof(float);
    return b;
}

namespace {

// Warp-aggregated accumulation of one value set per lane, keyed by window
// index (key < 0: no contribution). All 32 lanes must call it.
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

}  // namespace

namespace {

// Merge runs of equal keys among a lane's kPPT pixels, then reduce each run
// across the warp with a shuffle-driven key loop and add it to the global
// sums (all 32 lanes must call it).
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

// Assignment pass over one 32x32 tile.
//   FIRST: features come from the RGB bytes (and are stored for later passes).
//   LAST:  labels are written; otherwise every centre's member sums are
//          accumulated for the update (exact integers).
//   SAME:  S is a multiple of kPPT, so a thread's kPPT pixels share a cell.
template <bool FIRST, bool LAST, bool SAME>
__global__ void __launch_bounds__(kThreads, 3) k_assign(FrameArgs a, int store_feat) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = a.W, H = a.H, S = a.S;
    const int tx0 = blockIdx.x * kTileW, ty0 = blockIdx.y * kTileH;

    // Window of centres for this tile: the cells its pixels fall in plus one
    // ring.
    const int ccx0 = tx0 / S, ccx1 = min(tx0 + kTileW - 1, W - 1) / S;
    const int ccy0 = ty0 / S, ccy1 = min(ty0 + kTileH - 1, H - 1) / S;
    const int wx0 = ccx0 - 1, wy0 = ccy0 - 1;
    const int wnx = ccx1 - ccx0 + 3, wny = ccy1 - ccy0 + 3;
    const int nwin = wnx * wny;
    const bool direct = a.direct_acc != 0;

    float4 *cA = reinterpret_cast<float4 *>(smem_raw);
    float *cY = reinterpret_cast<float *>(cA + nwin);
    int *wacc = reinterpret_cast<int *>(smem_raw + (((size_t)a.win_max * 20 + 15) & ~(size_t)15));
    float *lut = reinterpret_cast<float *>(wacc + (direct ? 0 : (size_t)kWarps * a.win_max * 4));

    // Out-of-grid window cells hold a sentinel centre whose D is ~1e18, so
    // the candidate loop needs no bounds checks (the own cell is always
    // valid and always beats it).
    for (int i = tid; i < nwin; i += kThreads) {
        const int cy = wy0 + i / wnx, cx = wx0 + i - (i / wnx) * wnx;
        if (cx >= 0 && cx < a.ns_c && cy >= 0 && cy < a.ns_r) {
            const float *ck = a.centres + ((size_t)cy * a.ns_c + cx) * 6;
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
            wacc[q * a.win_max * 4 + (i - q * nwin * 4)] = 0;
        }
    }
    if (FIRST) {
        for (int i = tid; i < 256; i += kThreads) lut[i] = g_lut[i];
    }
    __syncthreads();

    const int x = tx0 + 16 * (warp & 1) + 4 * (lane & 3);
    const int y = ty0 + 8 * (warp >> 1) + (lane >> 2);
    const bool row_ok = (y < H) && (x < W);
    float f0[kPPT] = {}, f1[kPPT] = {}, f2[kPPT] = {};
    const size_t plane = (size_t)H * a.P;
    const size_t foff = (size_t)y * a.P + x;

    if (row_ok) {
        if (FIRST) {
            const uint8_t *p = a.rgb + ((size_t)y * W + x) * a.C;
            unsigned r[kPPT], g[kPPT], b[kPPT];
            if (a.rgb_vec && a.C == 3) {
                const uint32_t *q = reinterpret_cast<const uint32_t *>(p);
                const uint32_t w0 = __ldg(q), w1 = __ldg(q + 1), w2 = __ldg(q + 2);
                r[0] = w0 & 255; g[0] = (w0 >> 8) & 255; b[0] = (w0 >> 16) & 255; r[1] = w0 >> 24;
                g[1] = w1 & 255; b[1] = (w1 >> 8) & 255; r[2] = (w1 >> 16) & 255; g[2] = w1 >> 24;
                b[2] = w2 & 255; r[3] = (w2 >> 8) & 255; g[3] = (w2 >> 16) & 255; b[3] = w2 >> 24;
            } else if (a.rgb_vec) {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
                const uint32_t ws[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int j = 0; j < kPPT; ++j) {
                    r[j] = ws[j] & 255; g[j] = (ws[j] >> 8) & 255; b[j] = (ws[j] >> 16) & 255;
                }
            } else {
#pragma unroll
                for (int j = 0; j < kPPT; ++j) {
                    const bool ok = x + j < W;
                    r[j] = ok ? p[j * a.C + 0] : 0;
                    g[j] = ok ? p[j * a.C + 1] : 0;
                    b[j] = ok ? p[j * a.C + 2] : 0;
                }
            }
#pragma unroll
            for (int j = 0; j < kPPT; ++j) convert_pixel(a.conv, r[j], g[j], b[j], lut, f0[j], f1[j], f2[j]);
            if (!LAST || store_feat) {
                if ((a.P & 3) == 0) {
                    *reinterpret_cast<float4 *>(a.feat + foff) = make_float4(f0[0], f0[1], f0[2], f0[3]);
                    *reinterpret_cast<float4 *>(a.feat + plane + foff) = make_float4(f1[0], f1[1], f1[2], f1[3]);
                    *reinterpret_cast<float4 *>(a.feat + 2 * plane + foff) =
                        make_float4(f2[0], f2[1], f2[2], f2[3]);
                } else {
                    for (int j = 0; j < kPPT && x + j < W; ++j) {
                        a.feat[foff + j] = f0[j];
                        a.feat[plane + foff + j] = f1[j];
                        a.feat[2 * plane + foff + j] = f2[j];
                    }
                }
            }
        } else {
            if ((a.P & 3) == 0) {
                const float4 v0 = __ldg(reinterpret_cast<const float4 *>(a.feat + foff));
                const float4 v1 = __ldg(reinterpret_cast<const float4 *>(a.feat + plane + foff));
                const float4 v2 = __ldg(reinterpret_cast<const float4 *>(a.feat + 2 * plane + foff));
                f0[0] = v0.x; f0[1] = v0.y; f0[2] = v0.z; f0[3] = v0.w;
                f1[0] = v1.x; f1[1] = v1.y; f1[2] = v1.z; f1[3] = v1.w;
                f2[0] = v2.x; f2[1] = v2.y; f2[2] = v2.z; f2[3] = v2.w;
            } else {
#pragma unroll
                for (int j = 0; j < kPPT; ++j) {
                    const bool ok = x + j < W;
                    f0[j] = ok ? a.feat[foff + j] : 0.0f;
                    f1[j] = ok ? a.feat[plane + foff + j] : 0.0f;
                    f2[j] = ok ? a.feat[2 * plane + foff + j] : 0.0f;
                }
            }
        }
    }

    // Own cell of each pixel: column cx[j], row pcy.
    const int pcy = y / S;
    int cx[kPPT];
    {
        const int c0 = x / S;
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
        const float w = a.w;
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
                    bk[j] = min(bk[j], (__float_as_uint(D) & ~15u) | (unsigned)t);
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
            best[j] = ok ? (pcy + dy) * a.ns_c + cx[j] + dx : -1;
        else
            best[j] = ok ? (pcy + dy - wy0) * wnx + (cx[j] + dx - wx0) : -1;
    }

    if constexpr (LAST) {
        if (row_ok) {
            int32_t *out = a.labels + (size_t)y * W + x;
            if (a.labels_vec) {
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
        const float fs = a.fix_scale;
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
            unsigned *my = reinterpret_cast<unsigned *>(wacc) + (size_t)warp * a.win_max * 4;
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
            const unsigned *all = reinterpret_cast<const unsigned *>(wacc);
            for (int i = tid; i < nwin * 4; i += kThreads) {
                const int wi = i >> 2, c = i & 3;
                const int cy = wy0 + wi / wnx, cxg = wx0 + wi - (wi / wnx) * wnx;
                unsigned long long *g =
                    reinterpret_cast<unsigned long long *>(a.acc) + ((size_t)cy * a.ns_c + cxg) * 6;
                if (c < 3) {
                    long long t = 0;
#pragma unroll
                    for (int q = 0; q < kWarps; ++q) t += (int)all[(size_t)q * a.win_max * 4 + i];
                    if (t != 0) atomicAdd(&g[c], (unsigned long long)t);
                } else {
                    long long xs = 0, ys = 0, n = 0;
#pragma unroll
                    for (int q = 0; q < kWarps; ++q) {
                        const unsigned pk = all[(size_t)q * a.win_max * 4 + i];
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
            accumulate_runs(best, v, reinterpret_cast<unsigned long long *>(a.acc), wx0, wy0, wnx, a.ns_c);
        }
    }
}

// ---------------------------------------------------------------------------
// Update: centre = member mean; empty centre keeps position and colour.
// ---------------------------------------------------------------------------

__global__ void k_update(long long *acc, const float *centres_in, float *centres_out, int K, double fix_inv) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    long long *ak = acc + (size_t)k * 6;
    const long long n = ak[5];
    float *co = centres_out + (size_t)k * 6;
    const float *ci = centres_in + (size_t)k * 6;
    if (n > 0) {
        const double inv = 1.0 / (double)n;
        co[0] = (float)((double)ak[0] * fix_inv * inv);
        co[1] = (float)((double)ak[1] * fix_inv * inv);
        co[2] = (float)((double)ak[2] * fix_inv * inv);
        co[3] = (float)((double)ak[3] * inv);
        co[4] = (float)((double)ak[4] * inv);
        co[5] = (float)n;
    } else {
        if (co != ci) {
#pragma unroll
            for (int c = 0; c < 5; ++c) co[c] = ci[c];
        }
        co[5] = 0.0f;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) ak[c] = 0;
}

// Sums of the pixels of each label from an explicit label map (used for an
// update from given labels, e.g. a learned warm start). One thread per
// pixel; warp-aggregated global atomics.
__global__ void k_accumulate_labels(const float *feat, int W, int H, int P, const int32_t *labels, int K,
                                    long long *acc, float fs) {
    const int lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int x = (int)(i % W), y = (int)(i / W);
    int key = -1;
    int v[6] = {0, 0, 0, 0, 0, 0};
    if (i < (long long)W * H) {
        const int k = labels[i];
        if (k >= 0 && k < K) {
            const size_t plane = (size_t)H * P, off = (size_t)y * P + x;
            key = k;
            v[0] = __float2int_rn(feat[off] * fs);
            v[1] = __float2int_rn(feat[plane + off] * fs);
            v[2] = __float2int_rn(feat[2 * plane + off] * fs);
            v[3] = x;
            v[4] = y;
            v[5] = 1;
        }
    }
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

// ---------------------------------------------------------------------------
// Connectivity: one double-buffered pass.
// ---------------------------------------------------------------------------

__global__ void k_connectivity(const int32_t *__restrict__ in, int32_t *__restrict__ out, int W, int H) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        const size_t i = (size_t)y * W + x;
        const int32_t own = __ldg(in + i);
        int32_t nb[4];
        int n = 0;
        if (x > 0) nb[n++] = __ldg(in + i - 1);
        if (y > 0) nb[n++] = __ldg(in + i - W);
        if (x < W - 1) nb[n++] = __ldg(in + i + 1);
        if (y < H - 1) nb[n++] = __ldg(in + i + W);
        bool all_differ = n > 0;
        for (int j = 0; j < n; ++j) all_differ &= (nb[j] != own);
        int32_t result = own;
        if (all_differ) {
            int best_count = 0;
            for (int j = 0; j < n; ++j) {
                int cnt = 0;
                for (int q = 0; q < n; ++q) cnt += (nb[q] == nb[j]);
                if (cnt > best_count) {
                    best_count = cnt;
                    result = nb[j];
                }
            }
        }
        out[i] = result;
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------

cudaError_t upload_lut(const float *lut256) { return cudaMemcpyToSymbol(g_lut, lut256, 256 * sizeof(float)); }

template <bool F, bool L, bool SM>
static cudaError_t set_smem(int bytes) {
    return cudaFuncSetAttribute(k_assign<F, L, SM>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
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

cudaError_t launch_init_from_rgb(const FrameArgs &a, float *centres, cudaStream_t s) {
    const int K = a.ns_c * a.ns_r;
    k_init_rgb<<<(K + 127) / 128, 128, 0, s>>>(a, centres, a.acc);
    return cudaGetLastError();
}

cudaError_t launch_init_from_feat(const float *feat, int W, int H, int P, int S, int ns_c, int ns_r,
                                  float *centres, cudaStream_t s) {
    const int K = ns_c * ns_r;
    k_init_feat<<<(K + 127) / 128, 128, 0, s>>>(feat, W, H, P, S, ns_c, ns_r, centres);
    return cudaGetLastError();
}

cudaError_t launch_zero_acc(long long *acc, int K, cudaStream_t s) {
    const int n = K * 6;
    k_zero_acc<<<(n + 255) / 256, 256, 0, s>>>(acc, n);
    return cudaGetLastError();
}

cudaError_t launch_assign(const FrameArgs &a, bool first, bool last, bool store_feat, size_t smem,
                          cudaStream_t s) {
    const dim3 grid((a.W + kTileW - 1) / kTileW, (a.H + kTileH - 1) / kTileH);
    const int sf = store_feat ? 1 : 0;
    const bool same = (a.S % kPPT) == 0;
    if (same) {
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

cudaError_t launch_update(long long *acc, const float *centres_in, float *centres_out, int K, double fix_inv,
                          cudaStream_t s) {
    k_update<<<(K + 127) / 128, 128, 0, s>>>(acc, centres_in, centres_out, K, fix_inv);
    return cudaGetLastError();
}

cudaError_t launch_accumulate_labels(const float *feat, int W, int H, int P, const int32_t *labels, int K,
                                     long long *acc, float fix_scale, cudaStream_t s) {
    const long long n = (long long)W * H;
    k_accumulate_labels<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(feat, W, H, P, labels, K, acc, fix_scale);
    return cudaGetLastError();
}

static dim3 rows_grid(int W, int H, int bx) { return dim3((W + bx - 1) / bx, H < 65535 ? H : 65535); }

cudaError_t launch_convert(const ConvConsts &cc, const uint8_t *rgb, int W, int H, int C, float *feat, int P,
                           cudaStream_t s) {
    k_convert<<<rows_grid(W, H, 128), 128, 0, s>>>(cc, rgb, W, H, C, feat, P);
    return cudaGetLastError();
}

cudaError_t launch_connectivity(const int32_t *in, int32_t *out, int W, int H, cudaStream_t s) {
    k_connectivity<<<rows_grid(W, H, 128), 128, 0, s>>>(in, out, W, H);
    return cudaGetLastError();
}

}  // namespace slicgb
