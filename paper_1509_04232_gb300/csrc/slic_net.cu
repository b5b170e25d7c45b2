// Learned warm start: a 4-layer 3x3 convolutional network (C0=14 -> 32 -> 32
// -> 32 -> 9, ReLU between layers, zero padding) that predicts, for every
// pixel, logits over the 9 cells of its 3x3 cell window (slot t = (dy+1)*3 +
// (dx+1)). Weights and stored activations are bfloat16, every product sum is
// accumulated in FP32 on the 5th-generation tensor cores (tcgen05.mma with
// tensor-memory accumulators): the forward convolutions, the input gradients
// (the same kernel with mirrored taps) and the weight gradients. Training
// (softmax cross-entropy against the slots of reference labels, Adam with
// FP32 master weights) and inference run entirely in the kernels below;
// the C ABI is at the end of this file and declared in include/slic.h.
//
// Layouts: activations NHWC bf16 with the channel count padded to a multiple
// of 16 (layer-1 input 16, hidden 32, logits 16 in FP32). Weights per layer:
// master FP32 and gradients [9][Cin_p][Cout_p] (tap = dy*3 + dx), a bf16
// copy [9][Cout_p][Cin_p] for the forward pass and one [9][Cin_p][Cout_p]
// for the input-gradient pass: each the K-major operand (K = the input
// channels of its convolution) that the tensor-core kernel stages.
#include "slic.h"
#include "slic_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <utility>
#include <vector>

using namespace slicgb;

namespace {

__device__ float g_lut_net[256];  // sRGB byte -> linear (this file's copy)

cudaError_t net_upload_lut() {
    float t[256];
    srgb_table(t);
    return cudaMemcpyToSymbol(g_lut_net, t, sizeof t);
}

constexpr int kLayers = 4;
constexpr int kCinReal[kLayers] = {14, 32, 32, 32};
constexpr int kCoutReal[kLayers] = {32, 32, 32, 9};
constexpr int kCinPad[kLayers] = {16, 32, 32, 32};
constexpr int kCoutPad[kLayers] = {32, 32, 32, 16};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// max(lo, 0) and max(hi, 0) rounded to bf16 in one conversion (hi in the
// upper half).
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}


// Square root on the hardware approximation (relative error ~2^-22, far
// below the bf16 rounding of the channels).
__device__ __forceinline__ float sqrt_fast(float v) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// ---------------------------------------------------------------------------
// Input channels: L/100, a/128, b/128, (x mod S)/S, (y mod S)/S, then for the
// 9 slots of the pixel's cell window the Eq. (1) distance D/100 to the
// grid-initialised centre of that cell (2.0 off the grid), zero padding.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_net_prep(ConvConsts cc, const uint8_t *rgb, const uint8_t *const *table,
                                                  int W, int H, int C, int S, float w, __nv_bfloat16 *x0) {
    // A block covers 128 pixels of one row; the grid centres of the cells its
    // pixels see (three cell rows, the covered cell columns +- 1) are
    // converted once into shared memory instead of once per pixel and slot.
    constexpr int kMaxCols = 128 + 3;
    __shared__ float4 cen_lab[3][kMaxCols];  // L, a, b, x of a grid centre
    __shared__ float cen_y[3][kMaxCols];     // y (< 0: off the grid)
    const int x0p = blockIdx.x * blockDim.x, y = blockIdx.y, b = blockIdx.z;
    const size_t img = (size_t)b * H * W;
    // image b: entry b of the pointer table, else the b-th of a contiguous stack
    const uint8_t *const src = table ? table[b] : rgb + img * C;
    const int ns_c = (W + S - 1) / S, ns_r = (H + S - 1) / S;
    const int cy = y / S, cx_lo = x0p / S - 1;
    const int cx_hi = min(x0p + (int)blockDim.x - 1, W - 1) / S + 1;
    const int ncols = cx_hi - cx_lo + 1;
    for (int i = threadIdx.x; i < 3 * ncols; i += blockDim.x) {
        const int r = i / ncols, c = i - r * ncols;
        const int nx = cx_lo + c, ny = cy + r - 1;
        if (nx >= 0 && nx < ns_c && ny >= 0 && ny < ns_r) {
            // grid initialisation of Sec. 3: midpoint of the in-image cell, colour under it
            const int xf = nx * S, xl = min((nx + 1) * S, W) - 1, yf = ny * S, yl = min((ny + 1) * S, H) - 1;
            const uint8_t *q = src + ((size_t)((yf + yl) >> 1) * W + ((xf + xl) >> 1)) * C;
            float l, a2, b2;
            convert_pixel(cc, q[0], q[1], q[2], g_lut_net, l, a2, b2);
            cen_lab[r][c] = make_float4(l, a2, b2, 0.5f * (float)(xf + xl));
            cen_y[r][c] = 0.5f * (float)(yf + yl);
        } else {
            cen_lab[r][c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            cen_y[r][c] = -1.0f;
        }
    }
    __syncthreads();
    const int x = x0p + threadIdx.x;
    if (x >= W) return;
    const size_t px = img + (size_t)y * W + x;
    const uint8_t *p = src + ((size_t)y * W + x) * C;
    float f0, f1, f2;
    convert_pixel(cc, p[0], p[1], p[2], g_lut_net, f0, f1, f2);
    const int cx = x / S;
    const float inv_s = 1.0f / (float)S;
    float ch[16];
    ch[0] = f0 * 0.01f;
    ch[1] = f1 * (1.0f / 128.0f);
    ch[2] = f2 * (1.0f / 128.0f);
    ch[3] = (float)(x - cx * S) * inv_s;
    ch[4] = (float)(y - cy * S) * inv_s;
    const float fx = (float)x, fy = (float)y;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int col = cx + t % 3 - 1 - cx_lo;
        const float4 e = cen_lab[t / 3][col];
        const float ey = cen_y[t / 3][col];
        float d = 2.0f;
        if (ey >= 0.0f) {
            const float dl = e.x - f0, da = e.y - f1, db = e.z - f2;
            const float dx = e.w - fx, dy = ey - fy;
            d = (sqrt_fast(fmaf(dl, dl, fmaf(da, da, db * db))) + w * sqrt_fast(fmaf(dx, dx, dy * dy))) * 0.01f;
        }
        ch[5 + t] = d;
    }
    ch[14] = ch[15] = 0.0f;
    uint32_t out[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = pack_bf16(ch[2 * i], ch[2 * i + 1]);
    uint4 *dst = reinterpret_cast<uint4 *>(x0 + px * 16);
    dst[0] = make_uint4(out[0], out[1], out[2], out[3]);
    dst[1] = make_uint4(out[4], out[5], out[6], out[7]);
}

// ---------------------------------------------------------------------------
// Forward convolution on the 5th-generation tensor cores (tcgen05.mma, FP32
// accumulators in tensor memory), warp-specialised: one warp copies input
// tiles with the tensor-memory accelerator (TMA), one issues the MMAs, and
// the epilogue warps read the accumulators out (bias, activation, store).
// The roles meet on mbarrier rings: NS input stages (full / empty) and two
// accumulator buffers (full / empty).
//
// A work tile is 120 output pixels of one image row, 30 per TMEM lane
// quarter (epilogue warp q % 4). Quarter q's 32 MMA rows (positions) are
// x0-1+30q .. x0+30+30q, so the 30 outputs of a quarter need only its own
// rows; all CIN channels of a position form one row of CIN*2 bytes, copied
// with the 32-byte (CIN 16) or 64-byte (CIN 32) swizzle, zeros outside the
// image (the zero padding). For each kernel row dy one MMA chunk (M 128
// positions x N 3*COUT x K16) takes all three horizontal taps at once:
// column dx*COUT + co of the accumulator row of position q holds
// sum_dy,ci in[y+dy-1][q][ci] * w[dy][dx][co][ci], and the output at x is
// the sum over dx of column block dx at position x-1+dx (neighbouring lanes
// of one warp: two shuffles). Three times the N of a tap-by-tap loop, so
// each A row read from shared memory feeds three times the MACs. Weights
// [dy][dx*COUT+co][ci] use the K-major unswizzled canonical layout (8-row x
// 16-byte core matrices, leading offset = one 8-channel plane), staged once
// per CTA.
// ---------------------------------------------------------------------------
constexpr int kTcOut = 120;               // output pixels per tile
constexpr int kTcIn = 128;                // MMA rows (positions) per tile
constexpr int kTcSeg = 30;                // outputs per lane quarter
constexpr unsigned kTcWaitPolls = 1u << 20;

__device__ __forceinline__ unsigned tc_smem(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading
// (K-direction) and stride (M/N-direction) byte offsets, each >> 4 in 14
// bits, descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((unsigned long long)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// The same for a K-major operand whose rows (CIN*2 bytes) carry the 32- or
// 64-byte swizzle (layout type at bit 61: 6 or 4); the leading offset is
// unused there (one MMA's 32 bytes of K lie within a row).
__device__ __forceinline__ unsigned long long tc_desc_sw(unsigned addr, unsigned sbo, unsigned long long layout) {
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | (1ull << 16) |
           ((unsigned long long)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46) | (layout << 61);
}

// kind::f16 instruction descriptor: FP32 D, bf16 A and B (both K-major),
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr unsigned tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ bool tc_wait(unsigned long long *bar, unsigned parity) {
    for (unsigned i = 0; i < kTcWaitPolls; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(tc_smem(bar)), "r"(parity), "r"(1000u)
            : "memory");
        if (done) return true;
    }
    return false;
}

// NCOL (16 or 32) consecutive FP32 columns of this warp's 32 TMEM lanes,
// without the wait (tcgen05.wait::ld follows a batch of these).
template <int NCOL>
__device__ __forceinline__ void tc_ld_cols(unsigned taddr, float *v) {
    unsigned r[32];
    if constexpr (NCOL == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    }
#pragma unroll
    for (int i = 0; i < NCOL; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// Loss: masked softmax over the in-grid slots, cross-entropy against the
// target slot; writes dL/dlogits = (p - onehot) / n_total as bf16 [p][16]
// and accumulates the loss sum and the number of correct argmaxes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool slot_valid(int t, int cx, int cy, int ns_c, int ns_r) {
    const int nx = cx + t % 3 - 1, ny = cy + t / 3 - 1;
    return nx >= 0 && nx < ns_c && ny >= 0 && ny < ns_r;
}

// Shared memory of one forward-convolution CTA (plus 1 KB for aligning the
// stages to the swizzle pattern), its TMEM columns and epilogue warps (each
// takes 16 output channels of one lane quarter).
__host__ __device__ constexpr int tc_box_bytes(int cin) { return 3 * kTcIn * cin * 2; }
__host__ __device__ constexpr int tc_buf_cols(int cout) { return 3 * cout <= 64 ? 64 : 128; }
__host__ __device__ constexpr int tc_epi_warps(int cout) { return cout / 16 * 4; }
__host__ __device__ constexpr int tc_smem_bytes(int cin, int cout, bool staged, int ns) {
    return 1024 + ns * tc_box_bytes(cin) + 3 * (cin / 8) * 3 * cout * 16 + (staged ? tc_epi_warps(cout) * 32 * 32 : 0) +
           (2 * ns + 5) * 8 + 16;
}

// Bounded mbarrier wait that also gives up once another role has aborted.
__device__ __forceinline__ bool tc_wait_ab(unsigned long long *bar, unsigned parity, const volatile int *abort) {
    for (unsigned i = 0; i < kTcWaitPolls; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(tc_smem(bar)), "r"(parity), "r"(1000u)
            : "memory");
        if (done) return true;
        if (*abort) return false;
    }
    return false;
}

__device__ __forceinline__ void tc_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem(bar)) : "memory");
}

// BWD: the same convolution as the input gradient of a layer (Cout -> Cin):
// the input is the layer's dZ, the weights are its [tap][ci][co] copy taken
// with the tap mirrored (dA[y][x][ci] = sum over dy, dx, co of
// dZ[y+dy-1][x+dx-1][co] w[2-dy][2-dx][co][ci]), no bias, and the epilogue
// multiplies by the ReLU derivative of the previous layer's stored output
// (mask > 0) before the bf16 store: the result is the previous layer's dZ.
template <int CIN, int COUT, bool RELU, bool OUTF32, bool LABELS, int NS, bool BWD = false>
__global__ void __launch_bounds__((tc_epi_warps(COUT) + 2) * 32) k_conv_fwd_tc(
    const __grid_constant__ CUtensorMap in_map, const __nv_bfloat16 *wf, const float *bias, void *out, int W, int H,
    int n_img, int S, int *err, const __nv_bfloat16 *mask) {
    constexpr int NP = CIN / 8;                   // 8-channel planes
    constexpr int KC = CIN / 16;                  // K chunks per kernel row
    constexpr int ROWB = CIN * 2;                 // bytes of one staged position
    constexpr unsigned BOX = tc_box_bytes(CIN);   // bytes of one stage (12 copies of 32 positions)
    constexpr int NN = 3 * COUT;                  // MMA N: three horizontal taps x COUT
    constexpr int W_PLANE = NN * 16;              // bytes of one 8-channel weight plane
    constexpr int W_BYTES = 3 * NP * W_PLANE;
    constexpr unsigned long long LAYOUT = CIN == 32 ? 4ull : 6ull;  // 64- or 32-byte swizzle
    constexpr bool STAGED = !OUTF32 && !LABELS;   // bf16 activations leave through shared memory
    constexpr int BUFC = tc_buf_cols(COUT);       // TMEM columns per accumulator buffer
    constexpr int EW = tc_epi_warps(COUT);        // epilogue warps: 16 channels x one lane quarter each
    constexpr int NT = (EW + 2) * 32;
    constexpr int PRODUCER = EW, ISSUER = EW + 1; // warp roles
    static_assert(BOX % 1024 == 0, "stages must keep the swizzle pattern aligned");
    static_assert(!STAGED || COUT == 32, "staged stores assume 64-byte output pixels");
    static_assert(!BWD || (STAGED && !RELU), "the input gradient leaves as masked bf16");
    extern __shared__ __align__(16) unsigned char tc_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned char *in_s = sm;                     // [NS][dy][128 positions][ROWB]
    unsigned char *w_s = in_s + NS * BOX;
    unsigned char *o_s = w_s + W_BYTES;           // [EW][32 pixels][32 bytes] when STAGED
    unsigned long long *full = reinterpret_cast<unsigned long long *>(o_s + (STAGED ? EW * 32 * 32 : 0));
    unsigned long long *empty = full + NS;
    unsigned long long *tfull = empty + NS;       // [2] accumulators ready
    unsigned long long *tempty = tfull + 2;       // [2] accumulators read out (EW warps)
    unsigned long long *done = tempty + 2;        // every MMA of this CTA complete
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(done + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // Weights once per CTA: plane (dy, ci / 8), row dx * COUT + co holds
    // w[dy][dx][co][ci .. ci+7] (global [tap][co][ci], tap = dy * 3 + dx;
    // BWD: global row (8 - tap) * COUT + co).
    for (int i = tid; i < 3 * NN * NP; i += NT) {
        const int pl = i % NP, r = i / NP;  // r = dy * NN + dx * COUT + co
        const int dy = r / NN, n = r - dy * NN;
        const int src = BWD ? (8 - (dy * 3 + n / COUT)) * COUT + n % COUT : r;
        const uint4 v = *reinterpret_cast<const uint4 *>(wf + (size_t)src * CIN + pl * 8);
        *reinterpret_cast<uint4 *>(w_s + (dy * NP + pl) * W_PLANE + n * 16) = v;
    }
    if (tid == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&in_map)) : "memory");
        for (int i = 0; i < 2 * NS; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&full[i])));
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&tfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&tempty[i])), "n"(EW));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(done)));
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == ISSUER) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(tmem_slot)),
                     "n"(2 * BUFC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // generic-proxy writes (weights) -> visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;
    const unsigned tiles_x = (unsigned)((W + kTcOut - 1) / kTcOut);
    const unsigned total = (unsigned)n_img * (unsigned)H * tiles_x;  // < 2^31 (pixels < 2^31)
    const unsigned G = gridDim.x;
    auto fail = [&]() {
        *abort = 1;
        atomicOr(err, 1);
    };

    if (warp == PRODUCER) {
        // ---- producer: 12 tensor-map copies (4 quarters x 3 rows) per stage ----
        if (lane == 0) {
            int s = 0;
            unsigned u = 0;       // completed rounds of the ring
            unsigned issued = 0;  // bit s: a copy was issued into stage s
            unsigned lastpar = 0; // bit s: parity of that copy's completion
            for (unsigned t = blockIdx.x; t < total; t += G) {
                if (u > 0 && !tc_wait_ab(&empty[s], (u - 1) & 1u, abort)) {
                    fail();
                    break;
                }
                const unsigned tx = t % tiles_x, ry = t / tiles_x;
                const int y = (int)(ry % (unsigned)H), img = (int)(ry / (unsigned)H);
                const unsigned b = tc_smem(&full[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(BOX) : "memory");
                const unsigned dst0 = tc_smem(in_s + s * BOX);
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        asm volatile(
                            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
                            "{%2, %3, %4, %5}], [%6];" ::"r"(dst0 + (unsigned)((dy * kTcIn + 32 * q) * ROWB)),
                            "l"(reinterpret_cast<uint64_t>(&in_map)), "r"(0),
                            "r"((int)tx * kTcOut - 1 + kTcSeg * q), "r"(y + dy - 1), "r"(img), "r"(b)
                            : "memory");
                    }
                }
                issued |= 1u << s;
                lastpar = (lastpar & ~(1u << s)) | ((u & 1u) << s);
                if (++s == NS) {
                    s = 0;
                    ++u;
                }
            }
            // every copy lands before the shared memory is released
            for (int k = 0; k < NS; ++k)
                if (issued & (1u << k)) tc_wait(&full[k], (lastpar >> k) & 1u);
        }
    } else if (warp == ISSUER) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const unsigned idesc = tc_idesc(kTcIn, NN);
            int s = 0;
            unsigned u = 0, j = 0;
            for (unsigned t = blockIdx.x; t < total; t += G, ++j) {
                const int bf = (int)(j & 1u);
                if (!tc_wait_ab(&full[s], u & 1u, abort) ||
                    (j >= 2 && !tc_wait_ab(&tempty[bf], ((j >> 1) - 1) & 1u, abort))) {
                    fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned a0 = tc_smem(in_s + s * BOX), b0 = tc_smem(w_s), d = tmem + (unsigned)(bf * BUFC);
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
                    for (int kc = 0; kc < KC; ++kc) {
                        const unsigned long long ad = tc_desc_sw(a0 + dy * kTcIn * ROWB + kc * 32, 8 * ROWB, LAYOUT);
                        const unsigned long long bd = tc_desc(b0 + (dy * NP + 2 * kc) * W_PLANE, W_PLANE, 128);
                        const unsigned acc = (dy | kc) != 0 ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tc_smem(&tfull[bf]))
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tc_smem(&empty[s]))
                             : "memory");
                if (++s == NS) {
                    s = 0;
                    ++u;
                }
            }
            // all MMAs (and their commits) complete before TMEM is released
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc_smem(done))
                         : "memory");
            tc_wait(done, 0);
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32*(w%4) .. +31, channels 16*(w/4) .. +15 ----
        const int quarter = warp & 3, c0 = (warp >> 2) * 16;
        float bv[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) bv[c] = !BWD && c0 + c < COUT ? bias[c0 + c] : 0.0f;
        unsigned j = 0;
        for (unsigned t = blockIdx.x; t < total; t += G, ++j) {
            const int bf = (int)(j & 1u);
            if (!__all_sync(0xffffffffu, tc_wait_ab(&tfull[bf], (j >> 1) & 1u, abort))) {
                if (lane == 0) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float d0[32], d1[32], d2[32];
            const unsigned ta = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(bf * BUFC + c0);
            tc_ld_cols<16>(ta, d0);
            tc_ld_cols<16>(ta + COUT, d1);
            tc_ld_cols<16>(ta + 2 * COUT, d2);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) tc_arrive(&tempty[bf]);
            // output of lane l (l < 30): positions l, l+1, l+2 of this quarter
            float v[16];
#pragma unroll
            for (int c = 0; c < 16; ++c)
                v[c] = (d0[c] + bv[c]) + __shfl_down_sync(0xffffffffu, d1[c], 1) +
                       __shfl_down_sync(0xffffffffu, d2[c], 2);

            const unsigned tx = t % tiles_x, ry = t / tiles_x;
            const int y = (int)(ry % (unsigned)H), img = (int)(ry / (unsigned)H);
            const int xw = (int)tx * kTcOut + kTcSeg * quarter;  // output pixel of lane 0
            const size_t row0 = (size_t)img * H * W + (size_t)y * W;
            if constexpr (BWD) {
                // ReLU derivative of the previous layer: its stored output > 0
                const int x = xw + lane;
                if (lane < kTcSeg && x < W) {
                    const uint4 *mp = reinterpret_cast<const uint4 *>(mask + (row0 + x) * COUT + c0);
                    const uint4 m0 = mp[0], m1 = mp[1];
                    const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const uint32_t h = (mw[c >> 1] >> (16 * (c & 1))) & 0xFFFFu;  // bf16 bits
                        if (!(__uint_as_float(h << 16) > 0.0f)) v[c] = 0.0f;
                    }
                }
            }
            if constexpr (STAGED) {
                // Each lane packs its pixel's 32 bytes (16 channels) into the
                // warp's staging rows (16-byte chunks swizzled by pixel
                // group, conflict-free); then each store instruction writes
                // 16 whole 32-byte sectors.
                unsigned char *ow = o_s + warp * (32 * 32);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    uint32_t w4[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) w4[h] = RELU ? pack_bf16_relu(v[8 * k + 2 * h], v[8 * k + 2 * h + 1])
                                                             : pack_bf16(v[8 * k + 2 * h], v[8 * k + 2 * h + 1]);
                    *reinterpret_cast<uint4 *>(ow + lane * 32 + ((k ^ ((lane >> 2) & 1)) << 4)) =
                        make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int pp = i * 16 + (lane >> 1), k = lane & 1;
                    const uint4 c = *reinterpret_cast<const uint4 *>(ow + pp * 32 + ((k ^ ((pp >> 2) & 1)) << 4));
                    if (pp < kTcSeg && xw + pp < W)
                        *reinterpret_cast<uint4 *>(static_cast<unsigned char *>(out) + (row0 + xw + pp) * 64 + c0 * 2 +
                                                   k * 16) = c;
                }
                __syncwarp();
            } else {
                const int x = xw + lane;
                if (lane < kTcSeg && x < W) {
                    const size_t px = row0 + x;
                    if constexpr (LABELS) {
                        // argmax of the valid slots' logits (first maximum in
                        // slot order), as the stand-alone label kernel on
                        // stored logits
                        const int cx = x / S, cy = y / S, ns_c = (W + S - 1) / S, ns_r = (H + S - 1) / S;
                        float mx = -INFINITY;
                        int arg = 4;
#pragma unroll
                        for (int q = 0; q < 9; ++q) {
                            if (slot_valid(q, cx, cy, ns_c, ns_r) && v[q] > mx) {
                                mx = v[q];
                                arg = q;
                            }
                        }
                        static_cast<int32_t *>(out)[px] = (cy + arg / 3 - 1) * ns_c + cx + arg % 3 - 1;
                    } else {
                        float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(out) + px * COUT + c0);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float4 f = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                            if (RELU) {
                                f.x = fmaxf(f.x, 0.0f); f.y = fmaxf(f.y, 0.0f); f.z = fmaxf(f.z, 0.0f); f.w = fmaxf(f.w, 0.0f);
                            }
                            o[q] = f;
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == ISSUER) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(2 * BUFC));
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores: dW[dy*3+dx][ci][co] = sum over pixels
// (y, x) of a_in[y+dy-1][x+dx-1][ci] dZ[y][x][co] (zero outside the image).
// Kernel row dy has its own accumulator in tensor memory, D_dy[m][co] with
// m = dx*CIN + ci (rows from 3*CIN to 127 stay zero), fed by tcgen05.mma of
// M128 x N COUT x K16 over pixels: for output row y and the kWgK columns
// x0 .. of a work strip, A_dy[m][k] = a_in[y+dy-1][x0+k+dx-1][ci] and
// B[co][k] = dZ[y][x0+k][co], both K-major in the unswizzled canonical
// layout (planes of 8 pixels, one 16-byte row per m or co: the forward
// kernel's weight layout).
//
// A CTA walks strips of kWgK columns by kWgBand rows. Each input row is
// staged once (16-byte loads of its NHWC row with a one-pixel halo) and
// transposed into one of four row slots; output row y then reads the slots
// of rows y-1, y, y+1 as A_0, A_1, A_2 and its dZ row from one of two B
// slots, so a row costs one input-row and one dZ-row transposition. One
// thread issues the 3 x kWgK/16 MMAs of a row; a slot is refilled once the
// MMAs that read it have completed (tcgen05.commit on an mbarrier). Each CTA
// writes its partial dW once; k_reduce_partials adds them.
// ---------------------------------------------------------------------------
constexpr int kWgK = 64;     // pixels (columns) of a strip
constexpr int kWgBand = 32;  // rows of a strip
constexpr int kWgPlanes = kWgK / 8;
constexpr int kWgThreads = 256;
__host__ __device__ constexpr int wg_slot_bytes() { return kWgPlanes * 128 * 16; }
__host__ __device__ constexpr int wg_b_bytes(int cout) { return kWgPlanes * cout * 16; }
__host__ __device__ constexpr int wg_raw_a(int cin) { return (kWgK + 2) * cin * 2; }
__host__ __device__ constexpr int wg_raw_z(int cout) { return kWgK * cout * 2; }
__host__ __device__ constexpr int wg_smem_bytes(int cin, int cout) {
    return 128 + 4 * wg_slot_bytes() + 2 * wg_b_bytes(cout) + wg_raw_a(cin) + wg_raw_z(cout) + 64;
}

// Two bf16 (as raw 16-bit patterns) in one 32-bit word, lo in the low half.
__device__ __forceinline__ uint32_t bf16_pair(const __nv_bfloat16 &lo, const __nv_bfloat16 &hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWgThreads) k_conv_bwd_weight_tc(const __nv_bfloat16 *a_in,
                                                                   const __nv_bfloat16 *dz, int W, int H, int n_img,
                                                                   float *partial, int *err) {
    constexpr int M_REAL = 3 * CIN;
    constexpr int A_PLANE = 128 * 16, B_PLANE = COUT * 16;
    constexpr int SLOT = wg_slot_bytes(), BSLOT = wg_b_bytes(COUT);
    constexpr int TCOLS = 128;  // tensor memory: the three accumulators of COUT columns
    static_assert(M_REAL <= 128 && 3 * COUT <= TCOLS && (COUT == 16 || COUT == 32) && CIN % 8 == 0,
                  "shapes of the weight-gradient kernel");
    extern __shared__ __align__(16) unsigned char wg_dyn[];
    unsigned char *slots =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(wg_dyn) + 127) & ~(uintptr_t)127);
    unsigned char *bslots = slots + 4 * SLOT;
    __nv_bfloat16 *ra = reinterpret_cast<__nv_bfloat16 *>(bslots + 2 * BSLOT);  // [kWgK+2][CIN]
    __nv_bfloat16 *rz = ra + wg_raw_a(CIN) / 2;                                 // [kWgK][COUT]
    unsigned long long *mma_done = reinterpret_cast<unsigned long long *>(rz + wg_raw_z(COUT) / 2);  // [2]
    unsigned long long *fin = mma_done + 2;
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(fin + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // the padding rows of A in every slot stay zero
    for (int i = tid; i < 4 * kWgPlanes * (128 - M_REAL); i += kWgThreads) {
        const int r = M_REAL + i % (128 - M_REAL), pl = i / (128 - M_REAL);  // pl = slot * planes + plane
        *reinterpret_cast<uint4 *>(slots + pl * A_PLANE + r * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mma_done[i])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(tmem_slot)),
                     "n"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    // the input row yy of image img at x0-1 .. x0+kWgK into ra (zeros outside)
    auto stage_row = [&](size_t base, int yy, int x0) {
        for (int i = tid; i < (kWgK + 2) * (CIN / 8); i += kWgThreads) {
            const int v8 = i % (CIN / 8), px = i / (CIN / 8), gx = x0 - 1 + px;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gx >= 0 && gx < W && yy >= 0 && yy < H)
                v = *reinterpret_cast<const uint4 *>(a_in + (base + (size_t)yy * W + gx) * CIN + v8 * 8);
            *reinterpret_cast<uint4 *>(ra + (size_t)px * CIN + v8 * 8) = v;
        }
    };
    // ra transposed into a row slot: rows m = dx*CIN + ci, planes of 8 pixels
    auto transpose_row = [&](int slot) {
        unsigned char *A = slots + slot * SLOT;
        for (int i = tid; i < kWgPlanes * M_REAL; i += kWgThreads) {
            const int m = i % M_REAL, j = i / M_REAL, dx = m / CIN, ci = m - dx * CIN;
            const __nv_bfloat16 *src = ra + (size_t)(8 * j + dx) * CIN + ci;
            *reinterpret_cast<uint4 *>(A + j * A_PLANE + m * 16) =
                make_uint4(bf16_pair(src[0], src[CIN]), bf16_pair(src[2 * CIN], src[3 * CIN]),
                           bf16_pair(src[4 * CIN], src[5 * CIN]), bf16_pair(src[6 * CIN], src[7 * CIN]));
        }
    };
    // the MMAs of output row `it` have completed (commits alternate on two barriers)
    auto row_done = [&](int j) -> bool { return tc_wait(&mma_done[j & 1], (j >> 1) & 1); };

    const int segs = (W + kWgK - 1) / kWgK, bands = (H + kWgBand - 1) / kWgBand;
    const long long units = (long long)n_img * segs * bands;
    int it = 0;  // output rows of this CTA so far
    bool ok = true;
    for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int seg = (int)(u % segs);
        const long long q = u / segs;
        const int band = (int)(q % bands), img = (int)(q / bands);
        const int x0 = seg * kWgK, y0 = band * kWgBand, y1 = min(y0 + kWgBand, H);
        const size_t base = (size_t)img * H * W;
        // the previous strip's MMAs read every slot: let them complete
        const bool w = (it < 1 || row_done(it - 1)) && (it < 2 || row_done(it - 2));
        if (!__syncthreads_and(w ? 1 : 0)) {
            ok = false;
            break;
        }
        // input rows y0-1 and y0 into slots 0 and 1 (row yy in slot (yy - y0 + 1) % 4)
        for (int p = 0; p < 2; ++p) {
            stage_row(base, y0 - 1 + p, x0);
            __syncthreads();
            transpose_row(p);
            __syncthreads();
        }
        for (int r = y0; r < y1; ++r, ++it) {
            // raw rows: input row r+1 (its slot held row r-3, read by row it-2),
            // dZ row r (B slot it % 2, read by row it-2)
            stage_row(base, r + 1, x0);
            for (int i = tid; i < kWgK * (COUT / 8); i += kWgThreads) {
                const int v8 = i % (COUT / 8), px = i / (COUT / 8), gx = x0 + px;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (gx < W) v = *reinterpret_cast<const uint4 *>(dz + (base + (size_t)r * W + gx) * COUT + v8 * 8);
                *reinterpret_cast<uint4 *>(rz + px * COUT + v8 * 8) = v;
            }
            const bool w2 = r - y0 < 2 || row_done(it - 2);
            if (!__syncthreads_and(w2 ? 1 : 0)) {  // (also: the raw rows are complete)
                ok = false;
                break;
            }
            const int sn = (r - y0 + 2) & 3;
            transpose_row(sn);
            unsigned char *B = bslots + (it & 1) * BSLOT;
            for (int i = tid; i < kWgPlanes * COUT; i += kWgThreads) {
                const int co = i % COUT, j = i / COUT;
                const __nv_bfloat16 *src = rz + (size_t)(8 * j) * COUT + co;
                *reinterpret_cast<uint4 *>(B + j * B_PLANE + co * 16) =
                    make_uint4(bf16_pair(src[0], src[COUT]), bf16_pair(src[2 * COUT], src[3 * COUT]),
                               bf16_pair(src[4 * COUT], src[5 * COUT]), bf16_pair(src[6 * COUT], src[7 * COUT]));
            }
            // generic-proxy writes -> visible to the tensor core
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned idesc = tc_idesc(128, COUT);
                const unsigned b0 = tc_smem(B);
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    const unsigned a0 = tc_smem(slots + ((r - y0 + dy) & 3) * SLOT);  // input row r-1+dy
#pragma unroll
                    for (int kc = 0; kc < kWgK / 16; ++kc) {
                        const unsigned long long ad = tc_desc(a0 + 2 * kc * A_PLANE, A_PLANE, 128);
                        const unsigned long long bd = tc_desc(b0 + 2 * kc * B_PLANE, B_PLANE, 128);
                        const unsigned acc = (it > 0 || kc > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                tmem + (unsigned)(dy * COUT)),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tc_smem(&mma_done[it & 1]))
                             : "memory");
            }
        }
    }
    // every MMA complete, then each accumulator row out: warp w (< 4) reads
    // lanes 32w .. 32w+31 (rows m), columns dy*COUT .. +COUT-1
    if (tid == 0)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(fin))
                     : "memory");
    const bool f_ok = tc_wait(fin, 0);
    if (!__syncthreads_and(f_ok ? 1 : 0)) ok = false;
    if (!ok && tid == 0) atomicOr(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp < 4) {
        const int m = warp * 32 + lane;
        const int dx = m / CIN, ci = m - dx * CIN;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            float v[COUT];
            tc_ld_cols<COUT>(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(dy * COUT), v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < M_REAL) {
                float4 *dst = reinterpret_cast<float4 *>(partial +
                                                         (((size_t)blockIdx.x * 9 + dy * 3 + dx) * CIN + ci) * COUT);
#pragma unroll
                for (int q = 0; q < COUT / 4; ++q)
                    dst[q] = it > 0 ? make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3])
                                    : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TCOLS));
    }
}

__global__ void k_reduce_partials(const float *partial, int n_blocks, int n, float *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int b = 0; b < n_blocks; ++b) s += partial[(size_t)b * n + i];
    out[i] = s;
}

// Bias gradient: db[co] = sum_p dZ[p][co] (per-CTA sums, then atomics).
template <int COUT>
__global__ void k_bias_grad(const __nv_bfloat16 *dz, long long n_px, float *db) {
    __shared__ float s[COUT];
    if (threadIdx.x < COUT) s[threadIdx.x] = 0.0f;
    __syncthreads();
    const int co = threadIdx.x % COUT;
    float acc = 0.0f;
    for (long long p = (long long)blockIdx.x * (blockDim.x / COUT) + threadIdx.x / COUT; p < n_px;
         p += (long long)gridDim.x * (blockDim.x / COUT))
        acc += __bfloat162float(dz[p * COUT + co]);
    atomicAdd(&s[co], acc);
    __syncthreads();
    if (threadIdx.x < COUT) atomicAdd(&db[threadIdx.x], s[threadIdx.x]);
}


__global__ void k_softmax_ce(const float *logits, const uint8_t *target, int W, int H, int n_img, int S,
                             float inv_total, __nv_bfloat16 *dz, float *stats) {
    const long long n_px = (long long)W * H * n_img;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float loss = 0.0f, correct = 0.0f;
    if (p < n_px) {
        const int x = (int)(p % W), y = (int)((p / W) % H);
        const int cx = x / S, cy = y / S, ns_c = (W + S - 1) / S, ns_r = (H + S - 1) / S;
        const float *l = logits + p * 16;
        float mx = -INFINITY;
        int arg = 0;
        for (int t = 0; t < 9; ++t)
            if (slot_valid(t, cx, cy, ns_c, ns_r) && l[t] > mx) {
                mx = l[t];
                arg = t;
            }
        float e[9], sum = 0.0f;
        for (int t = 0; t < 9; ++t) {
            e[t] = slot_valid(t, cx, cy, ns_c, ns_r) ? __expf(l[t] - mx) : 0.0f;
            sum += e[t];
        }
        const int tg = target[p];
        loss = -(l[tg] - mx - __logf(sum));
        correct = (arg == tg) ? 1.0f : 0.0f;
        uint32_t g[8];
        for (int t = 0; t < 16; t += 2) {
            const float g0 = t < 9 ? (e[t] / sum - (t == tg ? 1.0f : 0.0f)) * inv_total : 0.0f;
            const float g1 = t + 1 < 9 ? (e[t + 1] / sum - (t + 1 == tg ? 1.0f : 0.0f)) * inv_total : 0.0f;
            g[t / 2] = pack_bf16(g0, g1);
        }
        uint4 *d = reinterpret_cast<uint4 *>(dz + p * 16);
        d[0] = make_uint4(g[0], g[1], g[2], g[3]);
        d[1] = make_uint4(g[4], g[5], g[6], g[7]);
    }
    for (int off = 16; off > 0; off >>= 1) {
        loss += __shfl_xor_sync(0xFFFFFFFFu, loss, off);
        correct += __shfl_xor_sync(0xFFFFFFFFu, correct, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&stats[0], loss);
        atomicAdd(&stats[1], correct);
    }
}

// Argmax over the in-grid slots -> label of the chosen cell.
__global__ void k_net_labels(const float *logits, int W, int H, int n_img, int S, int32_t *labels) {
    const long long n_px = (long long)W * H * n_img;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_px) return;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const int cx = x / S, cy = y / S, ns_c = (W + S - 1) / S, ns_r = (H + S - 1) / S;
    const float *l = logits + p * 16;
    float mx = -INFINITY;
    int arg = 4;
    for (int t = 0; t < 9; ++t)
        if (slot_valid(t, cx, cy, ns_c, ns_r) && l[t] > mx) {
            mx = l[t];
            arg = t;
        }
    labels[p] = (cy + arg / 3 - 1) * ns_c + cx + arg % 3 - 1;
}

// Training targets: the slot (dy+1)*3 + (dx+1) of each pixel's label
// relative to its own cell; 255 (and a count in *bad) for a label outside
// the pixel's 3x3 cell window.
__global__ void k_net_slots(const int32_t *labels, int W, int H, int n_img, int S, uint8_t *slots, int *bad) {
    const long long n_px = (long long)W * H * n_img;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_px) return;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const int ns_c = (W + S - 1) / S, ns_r = (H + S - 1) / S;
    const int k = labels[p];
    const int dx = k % ns_c - x / S, dy = k / ns_c - y / S;
    const bool ok = k >= 0 && k < ns_c * ns_r && dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1;
    slots[p] = ok ? (uint8_t)((dy + 1) * 3 + dx + 1) : (uint8_t)255;
    if (!ok && bad) atomicAdd(bad, 1);
}

// Adam on the FP32 master weights of one layer (padded layout; padding stays
// zero), refreshing both bf16 copies.
__global__ void k_adam(float *w, float *m, float *v, const float *g, int cin_p, int cout_p, int cin_r, int cout_r,
                       float lr, float b1, float b2, float eps, float c1, float c2, __nv_bfloat16 *wf,
                       __nv_bfloat16 *wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * cin_p * cout_p) return;
    const int co = i % cout_p, ci = (i / cout_p) % cin_p, tap = i / (cout_p * cin_p);
    float wi = w[i];
    if (ci < cin_r && co < cout_r) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        wi -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
    }
    const __nv_bfloat16 q = __float2bfloat16_rn(wi);
    wb[i] = q;
    wf[((size_t)tap * cout_p + co) * cin_p + ci] = q;
}

__global__ void k_adam_bias(float *b, float *m, float *v, const float *g, int cout_r, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int i = threadIdx.x;
    if (i >= cout_r) return;
    const float mi = b1 * m[i] + (1.0f - b1) * g[i];
    const float vi = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    b[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// bf16 copies from the FP32 master weights (after loading weights).
__global__ void k_weight_copies(const float *w, int cin_p, int cout_p, __nv_bfloat16 *wf, __nv_bfloat16 *wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * cin_p * cout_p) return;
    const int co = i % cout_p, ci = (i / cout_p) % cin_p, tap = i / (cout_p * cin_p);
    const __nv_bfloat16 q = __float2bfloat16_rn(w[i]);
    wb[i] = q;
    wf[((size_t)tap * cout_p + co) * cin_p + ci] = q;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct slic_net_ctx {
    int max_batch = 0, H = 0, W = 0, S = 0, device = 0;
    float m = 10.0f;
    long long step = 0;
    // per layer: master w [9][cin_p][cout_p], m, v, grad; bias (cout_p) + m, v, grad; bf16 copies
    float *w[kLayers] = {}, *wm[kLayers] = {}, *wv[kLayers] = {}, *wg[kLayers] = {};
    float *b[kLayers] = {}, *bm[kLayers] = {}, *bv[kLayers] = {}, *bg[kLayers] = {};
    __nv_bfloat16 *wf[kLayers] = {}, *wb[kLayers] = {};
    // activations for max_batch images: x0 (16 ch), a1..a3 (32 ch), logits (16 f32), dz buffers
    __nv_bfloat16 *act[kLayers] = {};
    float *logits = nullptr;
    __nv_bfloat16 *dzA = nullptr, *dzB = nullptr;
    float *partial = nullptr;
    int partial_blocks = 0;
    float *stats = nullptr;
    int *tc_err = nullptr;   // set by a timed-out wait of the tensor-core convolution
    // act[l] as a [max_batch][H][W][Cin_p] bf16 tensor, copied in 32 x Cin_p boxes
    // (32- or 64-byte swizzle) by the forward convolution of layer l
    CUtensorMap in_map[kLayers] = {};
    // the gradient buffers as inputs of the input-gradient convolutions:
    // dzA with 16 channels (dL/dlogits), dzB and dzA with 32
    CUtensorMap dz_map[3] = {};
    int sms = 0;
    ConvConsts conv{};
    std::string err;
    std::vector<void *> allocs;
};

namespace {

thread_local std::string g_net_error = "no error";

slic_status nfail(slic_net_ctx *n, slic_status st, const std::string &msg) {
    if (n)
        n->err = msg;
    else
        g_net_error = msg;
    return st;
}

template <typename T>
bool nalloc(slic_net_ctx *n, T **p, size_t count) {
    void *q = nullptr;
    if (dev_alloc(&q, sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    n->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return true;
}

size_t wcount(int l) { return (size_t)9 * kCinPad[l] * kCoutPad[l]; }

template <int CIN, int COUT, bool RELU, bool OUTF32, bool LABELS, int NS, bool BWD = false>
cudaError_t conv_fwd_tc(const CUtensorMap &in_map, const __nv_bfloat16 *wf, const float *b, void *out, int W, int H,
                        int n, int S, int *err, int sms, cudaStream_t s, const __nv_bfloat16 *mask = nullptr) {
    auto kern = k_conv_fwd_tc<CIN, COUT, RELU, OUTF32, LABELS, NS, BWD>;
    const int smem = tc_smem_bytes(CIN, COUT, !OUTF32 && !LABELS, NS);
    const int threads = (tc_epi_warps(COUT) + 2) * 32;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    // Persistent grid: as many CTAs per SM as registers (256-register warp
    // granules), shared memory (with the per-CTA reservation), warps and
    // TMEM (512 columns) allow.
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, smem_res = 0, regs_sm = 0, warps_sm = 0;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&warps_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e != cudaSuccess) return e;
    const int warps = threads / 32, warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    int per_sm = 512 / (2 * tc_buf_cols(COUT));
    per_sm = std::min(per_sm, smem_sm / (smem + smem_res));
    per_sm = std::min(per_sm, regs_sm / (warp_regs * warps));
    per_sm = std::min(per_sm, warps_sm / 32 / warps);
    per_sm = std::max(per_sm, 1);
    const long long tiles = (long long)n * H * ((W + kTcOut - 1) / kTcOut);
    const int grid = (int)(tiles < (long long)per_sm * sms ? tiles : (long long)per_sm * sms);
    kern<<<grid, threads, smem, s>>>(in_map, wf, b, out, W, H, n, S, err, mask);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t conv_bwd_weight_tc(const __nv_bfloat16 *a_in, const __nv_bfloat16 *dz, int W, int H, int n,
                               float *partial, int blocks, int *err, cudaStream_t s) {
    auto kern = k_conv_bwd_weight_tc<CIN, COUT>;
    const int smem = wg_smem_bytes(CIN, COUT);
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, kWgThreads, smem, s>>>(a_in, dz, W, H, n, partial, err);
    return cudaGetLastError();
}

// Layer l of the forward pass on the tensor cores, reading its input through
// the layer's tensor map. With `labels`, the last layer writes each pixel's
// label (argmax of its valid slots) instead of its logits.
cudaError_t conv_fwd(const slic_net_ctx *nc, int l, const __nv_bfloat16 *wf, const float *b, void *out, int W, int H,
                     int n, bool labels, cudaStream_t s) {
    const CUtensorMap &m = nc->in_map[l];
    if (l == 0) return conv_fwd_tc<16, 32, true, false, false, 4>(m, wf, b, out, W, H, n, nc->S, nc->tc_err, nc->sms, s);
    if (l < 3) return conv_fwd_tc<32, 32, true, false, false, 3>(m, wf, b, out, W, H, n, nc->S, nc->tc_err, nc->sms, s);
    if (labels)
        return conv_fwd_tc<32, 16, false, false, true, 3>(m, wf, b, out, W, H, n, nc->S, nc->tc_err, nc->sms, s);
    return conv_fwd_tc<32, 16, false, true, false, 3>(m, wf, b, out, W, H, n, nc->S, nc->tc_err, nc->sms, s);
}

// Forward pass into n->logits, or, with labels_out, straight to labels.
slic_status forward_all(slic_net_ctx *n, int batch, const uint8_t *d_images, cudaStream_t s,
                        int32_t *labels_out = nullptr, const uint8_t *const *d_table = nullptr, int C = 3) {
    const dim3 pg((n->W + 127) / 128, n->H, batch);
    k_net_prep<<<pg, 128, 0, s>>>(n->conv, d_images, d_table, n->W, n->H, C, n->S, n->m / (float)n->S, n->act[0]);
    cudaError_t e = cudaGetLastError();
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
        void *out = l < 3 ? static_cast<void *>(n->act[l + 1])
                          : (labels_out ? static_cast<void *>(labels_out) : static_cast<void *>(n->logits));
        e = conv_fwd(n, l, n->wf[l], n->b[l], out, n->W, n->H, batch, labels_out != nullptr, s);
    }
    if (e != cudaSuccess) return nfail(n, SLIC_ERR_CUDA, std::string("network forward launch: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

// Gradients of the mean cross-entropy for the batch into wg/bg (after forward_all).
slic_status backward_all(slic_net_ctx *n, int batch, const uint8_t *d_targets, cudaStream_t s) {
    const int W = n->W, H = n->H;
    const long long n_px = (long long)W * H * batch;
    cudaError_t e = cudaMemsetAsync(n->stats, 0, 2 * sizeof(float), s);
    if (e == cudaSuccess) {
        k_softmax_ce<<<(unsigned)((n_px + 255) / 256), 256, 0, s>>>(n->logits, d_targets, W, H, batch, n->S,
                                                                   1.0f / (float)n_px, n->dzA, n->stats);
        e = cudaGetLastError();
    }
    __nv_bfloat16 *dz = n->dzA, *dz_prev = n->dzB;
    for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
        const int cin = kCinPad[l], cout = kCoutPad[l];
        // weight gradient of layer l from its input act[l] and dz (per-CTA
        // partials on the tensor cores, then their sum)
        if (l == 0)
            e = conv_bwd_weight_tc<16, 32>(n->act[0], dz, W, H, batch, n->partial, n->partial_blocks, n->tc_err, s);
        else if (l < 3)
            e = conv_bwd_weight_tc<32, 32>(n->act[l], dz, W, H, batch, n->partial, n->partial_blocks, n->tc_err, s);
        else
            e = conv_bwd_weight_tc<32, 16>(n->act[l], dz, W, H, batch, n->partial, n->partial_blocks, n->tc_err, s);
        if (e != cudaSuccess) break;
        const int cnt = 9 * cin * cout;
        k_reduce_partials<<<(cnt + 255) / 256, 256, 0, s>>>(n->partial, n->partial_blocks, cnt, n->wg[l]);
        e = cudaMemsetAsync(n->bg[l], 0, sizeof(float) * cout, s);
        if (e != cudaSuccess) break;
        if (cout == 32)
            k_bias_grad<32><<<n->partial_blocks, 256, 0, s>>>(dz, n_px, n->bg[l]);
        else
            k_bias_grad<16><<<n->partial_blocks, 256, 0, s>>>(dz, n_px, n->bg[l]);
        e = cudaGetLastError();
        if (l > 0 && e == cudaSuccess) {
            // dz of layer l-1 (its output act[l] is layer l's input), on the
            // tensor cores: the forward convolution in its BWD form, reading
            // dz through its tensor map (dzA: 16 channels for l = 3, else 32)
            const CUtensorMap &m = n->dz_map[l == 3 ? 0 : (dz == n->dzB ? 1 : 2)];
            if (l < 3)
                e = conv_fwd_tc<32, 32, false, false, false, 3, true>(m, n->wb[l], nullptr, dz_prev, W, H, batch,
                                                                      n->S, n->tc_err, n->sms, s, n->act[l]);
            else
                e = conv_fwd_tc<16, 32, false, false, false, 4, true>(m, n->wb[l], nullptr, dz_prev, W, H, batch,
                                                                      n->S, n->tc_err, n->sms, s, n->act[l]);
            std::swap(dz, dz_prev);
        }
    }
    if (e != cudaSuccess) return nfail(n, SLIC_ERR_CUDA, std::string("network backward launch: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

}  // namespace

// The network as seen by the segmentation drivers (the learned warm start
// of slic_batch_set_warmstart / slic_set_warmstart).
bool slicgb::net_geometry(const slic_net_ctx *n, int *W, int *H, int *S, float *m, int *max_batch) {
    if (!n) return false;
    *W = n->W;
    *H = n->H;
    *S = n->S;
    *m = n->m;
    *max_batch = n->max_batch;
    return true;
}

// Labels of `batch` images into labels [batch][H][W], max_batch images per
// forward pass: image i is entry i of the device table d_table when given,
// else the i-th of the contiguous stack d_images (uint8 [H][W][C] each).
cudaError_t slicgb::net_forward_labels(slic_net_ctx *n, int batch, const uint8_t *d_images,
                                       const uint8_t *const *d_table, int C, int32_t *labels, cudaStream_t s) {
    const size_t px = (size_t)n->W * n->H;
    for (int b0 = 0; b0 < batch; b0 += n->max_batch) {
        const int nb = std::min(n->max_batch, batch - b0);
        const uint8_t *imgs = d_table ? nullptr : d_images + (size_t)b0 * px * C;
        if (forward_all(n, nb, imgs, s, labels + (size_t)b0 * px, d_table ? d_table + b0 : nullptr, C) != SLIC_OK)
            return cudaErrorLaunchFailure;
    }
    return cudaSuccess;
}

extern "C" {

slic_status slic_net_create(int max_batch, int width, int height, int S, float m, unsigned long long seed,
                            slic_net *out) {
    if (!out || max_batch <= 0 || width <= 0 || height <= 0 || S <= 0 || !(m >= 0.0f) ||
        (long long)width * height * max_batch >= (1LL << 31))
        return nfail(nullptr, SLIC_ERR_INVALID, "need out, max_batch, width, height, S > 0, m >= 0 and batch pixels < 2^31");
    *out = nullptr;
    slic_net_ctx *n = new (std::nothrow) slic_net_ctx;
    if (!n) return nfail(nullptr, SLIC_ERR_NOMEM, "host allocation failed");
    n->max_batch = max_batch;
    n->W = width;
    n->H = height;
    n->S = S;
    n->m = m;
    n->conv = conv_consts(SLIC_CIELAB);
    cudaError_t e = cudaGetDevice(&n->device);
    if (e == cudaSuccess) e = device_setup(n->device, 0);
    if (e == cudaSuccess) e = net_upload_lut();
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, n->device);
    if (e != cudaSuccess) {
        delete n;
        return nfail(nullptr, SLIC_ERR_CUDA, std::string("CUDA set-up: ") + cudaGetErrorString(e));
    }
    n->partial_blocks = 2 * sms;
    n->sms = sms;
    const size_t px = (size_t)width * height * max_batch;
    bool ok = true;
    for (int l = 0; l < kLayers && ok; ++l) {
        ok = nalloc(n, &n->w[l], wcount(l)) && nalloc(n, &n->wm[l], wcount(l)) && nalloc(n, &n->wv[l], wcount(l)) &&
             nalloc(n, &n->wg[l], wcount(l)) && nalloc(n, &n->b[l], kCoutPad[l]) && nalloc(n, &n->bm[l], kCoutPad[l]) &&
             nalloc(n, &n->bv[l], kCoutPad[l]) && nalloc(n, &n->bg[l], kCoutPad[l]) &&
             nalloc(n, &n->wf[l], wcount(l)) && nalloc(n, &n->wb[l], wcount(l)) &&
             nalloc(n, &n->act[l], px * kCinPad[l]);
    }
    ok = ok && nalloc(n, &n->logits, px * 16) && nalloc(n, &n->dzA, px * 32) && nalloc(n, &n->dzB, px * 32) &&
         nalloc(n, &n->partial, (size_t)n->partial_blocks * 9 * 32 * 32) && nalloc(n, &n->stats, 2) &&
         nalloc(n, &n->tc_err, 1) && cudaMemset(n->tc_err, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        slic_net_destroy(n);
        return nfail(nullptr, SLIC_ERR_NOMEM, "device allocation for the network failed");
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    for (int l = 0; l < kLayers && ok; ++l) {
        const cuuint64_t c = (cuuint64_t)kCinPad[l];
        const cuuint64_t dims[4] = {c, (cuuint64_t)width, (cuuint64_t)height, (cuuint64_t)max_batch};
        const cuuint64_t strides[3] = {c * 2, c * 2 * width, c * 2 * width * height};
        const cuuint32_t box[4] = {(cuuint32_t)c, 32, 1, 1};
        const cuuint32_t ones[4] = {1, 1, 1, 1};
        ok = enc && enc(&n->in_map[l], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, n->act[l], dims, strides, box, ones,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, c == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    for (int k = 0; k < 3 && ok; ++k) {
        const cuuint64_t c = k == 0 ? 16 : 32;
        const cuuint64_t dims[4] = {c, (cuuint64_t)width, (cuuint64_t)height, (cuuint64_t)max_batch};
        const cuuint64_t strides[3] = {c * 2, c * 2 * width, c * 2 * width * height};
        const cuuint32_t box[4] = {(cuuint32_t)c, 32, 1, 1};
        const cuuint32_t ones[4] = {1, 1, 1, 1};
        ok = enc(&n->dz_map[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, k == 1 ? n->dzB : n->dzA, dims, strides, box,
                 ones, CU_TENSOR_MAP_INTERLEAVE_NONE, c == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if (!ok) {
        slic_net_destroy(n);
        return nfail(nullptr, SLIC_ERR_CUDA, "tensor maps of the network activations could not be encoded");
    }
    // He-normal initialisation of the real weights (FP32 master), zero biases
    // and moments; padding stays zero.
    std::mt19937_64 rng(seed);
    for (int l = 0; l < kLayers; ++l) {
        std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / (9.0f * kCinReal[l])));
        std::vector<float> hw(wcount(l), 0.0f);
        for (int tap = 0; tap < 9; ++tap)
            for (int ci = 0; ci < kCinReal[l]; ++ci)
                for (int co = 0; co < kCoutReal[l]; ++co)
                    hw[((size_t)tap * kCinPad[l] + ci) * kCoutPad[l] + co] = nd(rng);
        e = cudaMemcpy(n->w[l], hw.data(), sizeof(float) * hw.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(n->wm[l], 0, sizeof(float) * wcount(l));
        if (e == cudaSuccess) e = cudaMemset(n->wv[l], 0, sizeof(float) * wcount(l));
        if (e == cudaSuccess) e = cudaMemset(n->b[l], 0, sizeof(float) * kCoutPad[l]);
        if (e == cudaSuccess) e = cudaMemset(n->bm[l], 0, sizeof(float) * kCoutPad[l]);
        if (e == cudaSuccess) e = cudaMemset(n->bv[l], 0, sizeof(float) * kCoutPad[l]);
        if (e == cudaSuccess) {
            k_weight_copies<<<(unsigned)((wcount(l) + 255) / 256), 256>>>(n->w[l], kCinPad[l], kCoutPad[l], n->wf[l],
                                                                        n->wb[l]);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        slic_net_destroy(n);
        return nfail(nullptr, SLIC_ERR_CUDA, std::string("network initialisation: ") + cudaGetErrorString(e));
    }
    *out = n;
    return SLIC_OK;
}

slic_status slic_net_destroy(slic_net n) {
    if (!n) return SLIC_OK;
    cudaDeviceSynchronize();
    for (void *p : n->allocs) cudaFree(p);
    delete n;
    return SLIC_OK;
}

slic_status slic_net_param_count(slic_net n, size_t *count) {
    if (!n || !count) return nfail(n, SLIC_ERR_INVALID, "NULL argument");
    size_t c = 0;
    for (int l = 0; l < kLayers; ++l) c += (size_t)9 * kCinReal[l] * kCoutReal[l] + kCoutReal[l];
    *count = c;
    return SLIC_OK;
}

slic_status slic_net_status(slic_net n) {
    if (!n) return nfail(nullptr, SLIC_ERR_INVALID, "NULL network");
    int flag = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag) e = cudaMemset(n->tc_err, 0, sizeof(int));
    if (e != cudaSuccess) return nfail(n, SLIC_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (flag) return nfail(n, SLIC_ERR_TIMEOUT, "a bounded wait in the tensor-core convolution timed out");
    return SLIC_OK;
}

// Host <-> device parameters in the order layer by layer, W[dy][dx][ci][co]
// then b[co], real (unpadded) sizes; FP32 master values. `which` 0 selects
// the weights, 1 the last computed gradients.
slic_status slic_net_get_params(slic_net n, int which, float *h_out, size_t count) {
    size_t need = 0;
    if (!n || !h_out || slic_net_param_count(n, &need) != SLIC_OK || count != need || (which != 0 && which != 1))
        return nfail(n, SLIC_ERR_INVALID, "bad arguments (count must equal slic_net_param_count)");
    cudaError_t e = cudaDeviceSynchronize();
    size_t off = 0;
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
        std::vector<float> hw(wcount(l)), hb(kCoutPad[l]);
        e = cudaMemcpy(hw.data(), which ? n->wg[l] : n->w[l], sizeof(float) * hw.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(hb.data(), which ? n->bg[l] : n->b[l], sizeof(float) * hb.size(), cudaMemcpyDeviceToHost);
        for (int tap = 0; tap < 9; ++tap)
            for (int ci = 0; ci < kCinReal[l]; ++ci)
                for (int co = 0; co < kCoutReal[l]; ++co)
                    h_out[off++] = hw[((size_t)tap * kCinPad[l] + ci) * kCoutPad[l] + co];
        for (int co = 0; co < kCoutReal[l]; ++co) h_out[off++] = hb[co];
    }
    if (e != cudaSuccess) return nfail(n, SLIC_ERR_CUDA, std::string("parameter read: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

slic_status slic_net_set_params(slic_net n, const float *h_in, size_t count) {
    size_t need = 0;
    if (!n || !h_in || slic_net_param_count(n, &need) != SLIC_OK || count != need)
        return nfail(n, SLIC_ERR_INVALID, "bad arguments (count must equal slic_net_param_count)");
    cudaError_t e = cudaDeviceSynchronize();
    size_t off = 0;
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
        std::vector<float> hw(wcount(l), 0.0f), hb(kCoutPad[l], 0.0f);
        for (int tap = 0; tap < 9; ++tap)
            for (int ci = 0; ci < kCinReal[l]; ++ci)
                for (int co = 0; co < kCoutReal[l]; ++co)
                    hw[((size_t)tap * kCinPad[l] + ci) * kCoutPad[l] + co] = h_in[off++];
        for (int co = 0; co < kCoutReal[l]; ++co) hb[co] = h_in[off++];
        e = cudaMemcpy(n->w[l], hw.data(), sizeof(float) * hw.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(n->b[l], hb.data(), sizeof(float) * hb.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            k_weight_copies<<<(unsigned)((wcount(l) + 255) / 256), 256>>>(n->w[l], kCinPad[l], kCoutPad[l], n->wf[l],
                                                                        n->wb[l]);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return nfail(n, SLIC_ERR_CUDA, std::string("parameter write: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

slic_status slic_net_forward(slic_net n, int batch, const uint8_t *d_images, float *d_logits, int32_t *d_labels,
                             void *stream) {
    if (!n) return nfail(nullptr, SLIC_ERR_INVALID, "NULL network");
    if (batch <= 0 || batch > n->max_batch || !d_images) return nfail(n, SLIC_ERR_INVALID, "bad batch or images");
    cudaStream_t s = (cudaStream_t)stream;
    if (d_labels && !d_logits) return forward_all(n, batch, d_images, s, d_labels);  // labels fused into the last layer
    slic_status st = forward_all(n, batch, d_images, s);
    if (st != SLIC_OK) return st;
    const long long n_px = (long long)n->W * n->H * batch;
    cudaError_t e = cudaSuccess;
    if (d_logits) e = cudaMemcpyAsync(d_logits, n->logits, sizeof(float) * 16 * n_px, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && d_labels) {
        k_net_labels<<<(unsigned)((n_px + 255) / 256), 256, 0, s>>>(n->logits, n->W, n->H, batch, n->S, d_labels);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return nfail(n, SLIC_ERR_CUDA, std::string("network output: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

slic_status slic_net_gradients(slic_net n, int batch, const uint8_t *d_images, const uint8_t *d_targets,
                               float *d_stats, void *stream) {
    if (!n) return nfail(nullptr, SLIC_ERR_INVALID, "NULL network");
    if (batch <= 0 || batch > n->max_batch || !d_images || !d_targets)
        return nfail(n, SLIC_ERR_INVALID, "bad batch, images or targets");
    cudaStream_t s = (cudaStream_t)stream;
    slic_status st = forward_all(n, batch, d_images, s);
    if (st == SLIC_OK) st = backward_all(n, batch, d_targets, s);
    if (st == SLIC_OK && d_stats) {
        cudaError_t e = cudaMemcpyAsync(d_stats, n->stats, 2 * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return nfail(n, SLIC_ERR_CUDA, std::string("stats copy: ") + cudaGetErrorString(e));
    }
    return st;
}

slic_status slic_net_train_step(slic_net n, int batch, const uint8_t *d_images, const uint8_t *d_targets, float lr,
                                float *d_stats, void *stream) {
    slic_status st = slic_net_gradients(n, batch, d_images, d_targets, d_stats, stream);
    if (st != SLIC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    n->step += 1;
    const float c1 = 1.0f - std::pow(b1, (float)n->step), c2 = 1.0f - std::pow(b2, (float)n->step);
    for (int l = 0; l < kLayers; ++l) {
        k_adam<<<(unsigned)((wcount(l) + 255) / 256), 256, 0, s>>>(n->w[l], n->wm[l], n->wv[l], n->wg[l], kCinPad[l],
                                                                  kCoutPad[l], kCinReal[l], kCoutReal[l], lr, b1, b2,
                                                                  eps, c1, c2, n->wf[l], n->wb[l]);
        k_adam_bias<<<1, 32, 0, s>>>(n->b[l], n->bm[l], n->bv[l], n->bg[l], kCoutReal[l], lr, b1, b2, eps, c1, c2);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(n, SLIC_ERR_CUDA, std::string("optimiser launch: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

slic_status slic_net_slots(slic_net n, int batch, const int32_t *d_labels, uint8_t *d_slots, int *d_bad,
                           void *stream) {
    if (!n) return nfail(nullptr, SLIC_ERR_INVALID, "NULL network");
    if (batch <= 0 || !d_labels || !d_slots) return nfail(n, SLIC_ERR_INVALID, "bad batch, labels or slots");
    const long long n_px = (long long)n->W * n->H * batch;
    if (n_px >= (1LL << 40)) return nfail(n, SLIC_ERR_INVALID, "batch too large");
    k_net_slots<<<(unsigned)((n_px + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_labels, n->W, n->H, batch, n->S,
                                                                                 d_slots, d_bad);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(n, SLIC_ERR_CUDA, std::string("slot kernel launch: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

const char *slic_net_last_error(slic_net n) { return n ? n->err.c_str() : g_net_error.c_str(); }

}  // extern "C"
