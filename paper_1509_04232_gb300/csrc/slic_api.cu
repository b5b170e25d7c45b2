// C ABI of libslicgb.so (declared and documented in include/slic.h).
//
// Host-side responsibilities: parameter validation, the grid of Sec. 2,
// the colour constants (computed here in double precision from the sRGB and
// CIE definitions, then rounded to float), device scratch ownership, the
// stage order of the Sec. 4 Perform_Segmentation listing, launch accounting
// and the optional per-kernel event timing.
#include "slic.h"
#include "slic_internal.cuh"

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

using namespace slicgb;

struct slic_ctx {
    slic_params p{};
    int S = 0, ns_c = 0, ns_r = 0, K = 0, P = 0;
    int device = 0;
    float *feat = nullptr;        // 3 planes [H][P]
    long long *acc = nullptr;     // [K][6]
    int32_t *lbl_tmp = nullptr;   // [H][W] connectivity ping-pong
    ConvState *cstate = nullptr;  // stopping-test state of the current run
    int *ccl = nullptr;           // component connectivity scratch (mode 2), and its error flag
    int *ccl_err = nullptr;
    float fix_scale = 0.0f;
    size_t smem_max = 0;
    ConvConsts conv{};
    const float *init_centres = nullptr;
    slic_net net = nullptr;       // learned warm start (slic_set_warmstart)
    long long launches = 0;
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    size_t ev_used = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_error = "no error";

slic_status fail(slic_ctx *h, slic_status st, const std::string &msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return st;
}

slic_status cuda_fail(slic_ctx *h, cudaError_t e, const char *what) {
    return fail(h, SLIC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// sRGB linearisation (IEC 61966-2-1) of every byte value.
void make_lut(float lut[256]) {
    for (int i = 0; i < 256; ++i) {
        const double v = i / 255.0;
        const double lin = v <= 0.04045 ? v / 12.92 : std::pow((v + 0.055) / 1.055, 2.4);
        lut[i] = (float)lin;
    }
}

// Linear sRGB -> XYZ (D65). For CIELAB each row is divided by the white
// point (the row sum, i.e. the XYZ of linear white); for XYZ output the
// rows are scaled by 100.
ConvConsts make_conv(int color_space) {
    static const double M[3][3] = {{0.4124564, 0.3575761, 0.1804375},
                                   {0.2126729, 0.7151522, 0.0721750},
                                   {0.0193339, 0.1191920, 0.9503041}};
    ConvConsts c{};
    for (int r = 0; r < 3; ++r) {
        const double white = M[r][0] + M[r][1] + M[r][2];
        for (int k = 0; k < 3; ++k) c.m[3 * r + k] = (float)(color_space == SLIC_XYZ ? 100.0 * M[r][k] : M[r][k] / white);
    }
    c.eps = (float)(216.0 / 24389.0);
    c.k_slope = (float)((24389.0 / 27.0) / 116.0);
    c.k_offset = (float)(16.0 / 116.0);
    c.color_space = color_space;
    return c;
}

std::mutex g_lut_mu;
std::vector<int> g_lut_devices;
std::vector<std::pair<int, size_t>> g_smem_set;  // device -> largest dynamic smem configured

// Raise (never lower) the dynamic shared-memory limit of the assignment
// kernels on this device, so handles with different S can coexist.
cudaError_t ensure_smem(int dev, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_lut_mu);
    for (auto &d : g_smem_set)
        if (d.first == dev) {
            if (d.second >= bytes) return cudaSuccess;
            cudaError_t e = configure_kernels(bytes);
            if (e == cudaSuccess) d.second = bytes;
            return e;
        }
    cudaError_t e = configure_kernels(bytes);
    if (e == cudaSuccess) g_smem_set.emplace_back(dev, bytes);
    return e;
}

cudaError_t ensure_lut(int dev) {
    std::lock_guard<std::mutex> lk(g_lut_mu);
    for (int d : g_lut_devices)
        if (d == dev) return cudaSuccess;
    float lut[256];
    make_lut(lut);
    cudaError_t e = upload_lut(lut);
    if (e == cudaSuccess) g_lut_devices.push_back(dev);
    return e;
}

}  // namespace

namespace {
// Fault injection (SLIC_FAULT_ALLOC): the device allocation that takes this
// countdown from 1 to 0 fails; 0 means none.
std::atomic<long long> g_fail_allocs{0};
}  // namespace

namespace slicgb {
cudaError_t dev_malloc(void **p, size_t bytes) {
    long long n = g_fail_allocs.load();
    while (n > 0 && !g_fail_allocs.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
ConvConsts conv_consts(int color_space) { return make_conv(color_space); }
void srgb_table(float lut[256]) { make_lut(lut); }
cudaError_t device_setup(int dev, size_t smem) {
    cudaError_t e = ensure_lut(dev);
    if (e == cudaSuccess) e = ensure_smem(dev, smem);
    return e;
}
}  // namespace slicgb

namespace {

FrameArgs frame_args(slic_ctx *h, const uint8_t *rgb, float *feat, int P, const float *centres, int32_t *labels) {
    FrameArgs a{};
    a.conv = h->conv;
    a.rgb = rgb;
    a.feat = feat;
    a.centres = centres;
    a.centres_out = const_cast<float *>(centres);
    a.acc = h->acc;
    a.labels = labels;
    a.W = h->p.width;
    a.H = h->p.height;
    a.P = P;
    a.C = h->p.in_channels;
    a.S = h->S;
    a.ns_c = h->ns_c;
    a.ns_r = h->ns_r;
    a.w = h->p.m / (float)h->S;
    a.s_mul = h->S <= 2048 ? (unsigned)((0x100000000ULL + (unsigned)h->S - 1) / (unsigned)h->S) : 0u;
    a.tiles_x = (h->p.width + kTileW - 1) / kTileW;
    a.win_max = assign_max_window(h->S, h->ns_c, h->ns_r);
    a.direct_acc = assign_direct_acc(a.win_max) ? 1 : 0;
    a.rgb_vec = (rgb && (h->p.width & 3) == 0 && ((uintptr_t)rgb & 15) == 0) ? 1 : 0;
    a.labels_vec = (labels && (h->p.width & 3) == 0 && ((uintptr_t)labels & 15) == 0) ? 1 : 0;
    a.fix_scale = h->fix_scale;
    a.perturb = h->p.perturb_seeds;
    return a;
}

}  // namespace

// Under stream capture a record must be external to become an event-record
// node of the graph; outside capture it is a plain record.
cudaError_t slicgb::record_profile_event(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cudaEventRecordWithFlags(ev, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                             : cudaEventRecordDefault);
}

namespace {

slic_status assign_launch(slic_ctx *h, const FrameArgs &a, bool first, bool last, bool store_feat, cudaStream_t s) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->profiling) {
        if (h->ev_used == h->events.size()) {
            cudaEvent_t x, y;
            if (cudaEventCreate(&x) != cudaSuccess || cudaEventCreate(&y) != cudaSuccess)
                return fail(h, SLIC_ERR_CUDA, "cudaEventCreate failed");
            h->events.emplace_back(x, y);
        }
        e0 = h->events[h->ev_used].first;
        e1 = h->events[h->ev_used].second;
        ++h->ev_used;
        if (record_profile_event(e0, s) != cudaSuccess) return fail(h, SLIC_ERR_CUDA, "profile event record failed");
    }
    cudaError_t e = launch_assign(a, first, last, store_feat, assign_smem_bytes(assign_max_window(h->S, h->ns_c, h->ns_r), first), s);
    if (e != cudaSuccess) return cuda_fail(h, e, "assignment kernel launch");
    ++h->launches;
    if (h->profiling && record_profile_event(e1, s) != cudaSuccess)
        return fail(h, SLIC_ERR_CUDA, "profile event record failed");
    return SLIC_OK;
}

}  // namespace

extern "C" {

slic_status slic_create(const slic_params *params, slic_handle *out) {
    if (!params || !out) return fail(nullptr, SLIC_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const slic_params &p = *params;
    if (p.width <= 0 || p.height <= 0 || p.width > (1 << 20) || p.height > (1 << 20) ||
        (long long)p.width * p.height >= (1LL << 31))
        return fail(nullptr, SLIC_ERR_INVALID, "width and height must be in [1, 2^20] with width*height < 2^31");
    if (p.S < 0 || (p.S == 0 && p.K <= 0)) return fail(nullptr, SLIC_ERR_INVALID, "need S > 0 or K > 0");
    if (!(p.m >= 0.0f) || !std::isfinite(p.m)) return fail(nullptr, SLIC_ERR_INVALID, "m must be finite and >= 0");
    if (p.iterations < 0) return fail(nullptr, SLIC_ERR_INVALID, "iterations must be >= 0");
    if (p.color_space < 0 || p.color_space > 2) return fail(nullptr, SLIC_ERR_INVALID, "unknown color_space");
    if (p.in_channels != 3 && p.in_channels != 4) return fail(nullptr, SLIC_ERR_INVALID, "in_channels must be 3 or 4");
    if (p.enforce_connectivity < 0 || p.enforce_connectivity > 2)
        return fail(nullptr, SLIC_ERR_INVALID, "enforce_connectivity must be 0, 1 or 2");
    if (p.perturb_seeds != 0 && p.perturb_seeds != 1)
        return fail(nullptr, SLIC_ERR_INVALID, "perturb_seeds must be 0 or 1");
    if (!(p.convergence >= 0.0f) || !std::isfinite(p.convergence))
        return fail(nullptr, SLIC_ERR_INVALID, "convergence must be finite and >= 0");

    slic_ctx *h = new (std::nothrow) slic_ctx;
    if (!h) return fail(nullptr, SLIC_ERR_NOMEM, "host allocation failed");
    h->p = p;
    int S = p.S;
    if (S == 0) {
        S = (int)std::lround(std::sqrt((double)p.width * (double)p.height / (double)p.K));
        if (S < 1) S = 1;
    }
    h->S = S;
    h->ns_c = (p.width + S - 1) / S;
    h->ns_r = (p.height + S - 1) / S;
    if ((long long)h->ns_c * h->ns_r > (1LL << 26)) {
        delete h;
        return fail(nullptr, SLIC_ERR_INVALID, "too many superpixels (K_eff > 2^26)");
    }
    h->K = h->ns_c * h->ns_r;
    h->P = (p.width + 3) & ~3;
    h->conv = make_conv(p.color_space);
    h->fix_scale = p.color_space == SLIC_RGB ? 1.0f : kFixScaleFrac;

    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = ensure_lut(h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, SLIC_ERR_CUDA, std::string("CUDA initialisation: ") + cudaGetErrorString(e));
    }
    const size_t npix = (size_t)p.width * p.height;
    if (dev_alloc(&h->feat, sizeof(float) * 3 * (size_t)p.height * h->P) != cudaSuccess ||
        dev_alloc(&h->acc, sizeof(long long) * 6 * (size_t)h->K) != cudaSuccess ||
        dev_alloc(&h->lbl_tmp, sizeof(int32_t) * npix) != cudaSuccess ||
        dev_alloc(&h->cstate, sizeof(ConvState)) != cudaSuccess ||
        cudaMemset(h->cstate, 0, sizeof(ConvState)) != cudaSuccess || dev_alloc(&h->ccl_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(h->ccl_err, 0, sizeof(int)) != cudaSuccess ||
        (p.enforce_connectivity == 2 && dev_alloc(&h->ccl, sizeof(int) * ccl_scratch_ints((long long)npix)) != cudaSuccess)) {
        cudaGetLastError();
        cudaFree(h->feat);
        cudaFree(h->acc);
        cudaFree(h->lbl_tmp);
        cudaFree(h->cstate);
        cudaFree(h->ccl_err);
        cudaFree(h->ccl);
        delete h;
        return fail(nullptr, SLIC_ERR_NOMEM, "device allocation of scratch failed");
    }
    h->smem_max = assign_smem_bytes(assign_max_window(S, h->ns_c, h->ns_r), true);
    e = ensure_smem(h->device, h->smem_max);
    if (e != cudaSuccess) {
        slic_destroy(h);
        return fail(nullptr, SLIC_ERR_CUDA, std::string("kernel configuration: ") + cudaGetErrorString(e));
    }
    *out = h;
    return SLIC_OK;
}

slic_status slic_destroy(slic_handle h) {
    if (!h) return SLIC_OK;
    cudaDeviceSynchronize();
    cudaFree(h->feat);
    cudaFree(h->acc);
    cudaFree(h->lbl_tmp);
    cudaFree(h->cstate);
    cudaFree(h->ccl);
    cudaFree(h->ccl_err);
    for (auto &ev : h->events) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    delete h;
    return SLIC_OK;
}

slic_status slic_grid(slic_handle h, int *S, int *ns_c, int *ns_r) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (S) *S = h->S;
    if (ns_c) *ns_c = h->ns_c;
    if (ns_r) *ns_r = h->ns_r;
    return SLIC_OK;
}

slic_status slic_iterations_run(slic_handle h, int *out) {
    if (!h || !out) return fail(h, SLIC_ERR_INVALID, "NULL argument");
    ConvState cs{};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&cs, h->cstate, sizeof(ConvState), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "reading the stopping-test state");
    *out = cs.iters;
    return SLIC_OK;
}

slic_status slic_set_init_centres(slic_handle h, const float *d_init) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    h->init_centres = d_init;
    return SLIC_OK;
}

slic_status slic_segment(slic_handle h, const uint8_t *d_image, int32_t *d_labels, float *d_centres, void *stream) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (!d_image || !d_labels || !d_centres) return fail(h, SLIC_ERR_INVALID, "NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->p.iterations;
    FrameArgs a = frame_args(h, d_image, h->feat, h->P, d_centres, d_labels);
    a.cstate = h->cstate;
    a.conv_eps = h->p.convergence;
    cudaError_t e;
    const bool warm = h->net != nullptr;
    if (warm) {
        // Learned warm start: features first, the grid (or armed) initial
        // centres, then the member means of the network's labels (written to
        // lbl_tmp, free until connectivity) by one plain update.
        e = launch_convert(h->conv, d_image, h->p.width, h->p.height, h->p.in_channels, h->feat, h->P, s);
        if (e == cudaSuccess) {
            if (h->init_centres)
                e = h->init_centres == d_centres
                        ? cudaSuccess
                        : cudaMemcpyAsync(d_centres, h->init_centres, sizeof(float) * 6 * (size_t)h->K,
                                          cudaMemcpyDeviceToDevice, s);
            else
                e = launch_init_from_feat(h->feat, h->p.width, h->p.height, h->P, h->S, h->ns_c, h->ns_r,
                                          h->p.perturb_seeds, d_centres, s);
        }
        h->init_centres = nullptr;
        if (e == cudaSuccess) e = cudaMemsetAsync(h->cstate, 0, sizeof(ConvState), s);
        if (e == cudaSuccess) e = launch_zero_acc(h->acc, h->K, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "warm-start set-up");
        if (net_forward_labels(h->net, 1, d_image, nullptr, h->p.in_channels, h->lbl_tmp, s) != cudaSuccess)
            return fail(h, SLIC_ERR_CUDA, std::string("network forward: ") + slic_net_last_error(h->net));
        e = launch_accumulate_labels(h->feat, h->p.width, h->p.height, h->P, h->lbl_tmp, h->K, h->acc, h->fix_scale, s);
        if (e == cudaSuccess)
            e = launch_update(h->acc, d_centres, d_centres, h->K, 1.0f / h->fix_scale, nullptr, 0.0f, 0, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "warm-start update");
        h->launches += 4;
    } else if (h->init_centres) {
        if (h->init_centres != d_centres) {
            e = cudaMemcpyAsync(d_centres, h->init_centres, sizeof(float) * 6 * (size_t)h->K,
                                cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy of initial centres");
        }
        h->init_centres = nullptr;
        e = launch_zero_acc(h->acc, h->K, s);
        // (the grid initialisation resets the stopping-test state itself)
        if (e == cudaSuccess) e = cudaMemsetAsync(h->cstate, 0, sizeof(ConvState), s);
    } else {
        e = launch_init_from_rgb(a, s);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "initialisation kernel launch");
    ++h->launches;
    for (int pass = 0; pass <= n; ++pass) {
        if (pass > 0) {
            e = launch_update(h->acc, d_centres, d_centres, h->K, 1.0f / h->fix_scale, h->cstate, h->p.convergence,
                              pass, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "update kernel launch");
            ++h->launches;
        }
        slic_status st = assign_launch(h, a, pass == 0 && !warm, pass == n, pass != n, s);
        if (st != SLIC_OK) return st;
    }
    if (h->p.enforce_connectivity == 1) {
        e = launch_connectivity(d_labels, h->lbl_tmp, h->p.width, h->p.height, s);
        if (e == cudaSuccess) e = launch_connectivity(h->lbl_tmp, d_labels, h->p.width, h->p.height, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "connectivity kernel launch");
        h->launches += 2;
    } else if (h->p.enforce_connectivity == 2) {
        e = launch_connectivity_components(d_labels, d_labels, h->p.width, h->p.height, h->S * h->S / 4, h->ccl,
                                           h->ccl_err, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "component connectivity launch");
        h->launches += 9;
    }
    return SLIC_OK;
}

slic_status slic_set_warmstart(slic_handle h, slic_net net) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (net) {
        int W = 0, H = 0, S = 0, max_batch = 0;
        float m = 0.0f;
        net_geometry(net, &W, &H, &S, &m, &max_batch);
        if (W != h->p.width || H != h->p.height || S != h->S || m != h->p.m)
            return fail(h, SLIC_ERR_INVALID, "the network was made for another width, height, S or m");
    }
    h->net = net;
    return SLIC_OK;
}

slic_status slic_convert(slic_handle h, const uint8_t *d_image, float *d_features, void *stream) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (!d_image || !d_features) return fail(h, SLIC_ERR_INVALID, "NULL buffer");
    cudaError_t e = launch_convert(h->conv, d_image, h->p.width, h->p.height, h->p.in_channels, d_features,
                                   h->p.width, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "conversion kernel launch");
    ++h->launches;
    return SLIC_OK;
}

slic_status slic_init_centres(slic_handle h, const float *d_features, float *d_centres, void *stream) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (!d_features || !d_centres) return fail(h, SLIC_ERR_INVALID, "NULL buffer");
    cudaError_t e = launch_init_from_feat(d_features, h->p.width, h->p.height, h->p.width, h->S, h->ns_c, h->ns_r,
                                          h->p.perturb_seeds, d_centres, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "initialisation kernel launch");
    ++h->launches;
    return SLIC_OK;
}

slic_status slic_assign(slic_handle h, const float *d_features, const float *d_centres, int32_t *d_labels,
                        void *stream) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (!d_features || !d_centres || !d_labels) return fail(h, SLIC_ERR_INVALID, "NULL buffer");
    if (((uintptr_t)d_features & 15) != 0)
        return fail(h, SLIC_ERR_INVALID, "features must be 16-byte aligned");
    FrameArgs a = frame_args(h, nullptr, const_cast<float *>(d_features), h->p.width, d_centres, d_labels);
    return assign_launch(h, a, false, true, false, (cudaStream_t)stream);
}

slic_status slic_update(slic_handle h, const float *d_features, const int32_t *d_labels, const float *d_centres_in,
                        float *d_centres_out, void *stream) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (!d_features || !d_labels || !d_centres_in || !d_centres_out) return fail(h, SLIC_ERR_INVALID, "NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_zero_acc(h->acc, h->K, s);
    if (e == cudaSuccess)
        e = launch_accumulate_labels(d_features, h->p.width, h->p.height, h->p.width, d_labels, h->K, h->acc,
                                     h->fix_scale, s);
    if (e == cudaSuccess)
        e = launch_update(h->acc, d_centres_in, d_centres_out, h->K, 1.0f / h->fix_scale, nullptr, 0.0f, 1, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "update kernel launch");
    h->launches += 3;
    return SLIC_OK;
}

slic_status slic_connectivity_pass(slic_handle h, const int32_t *d_in, int32_t *d_out, void *stream) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (!d_in || !d_out || d_in == d_out) return fail(h, SLIC_ERR_INVALID, "need distinct input and output");
    cudaError_t e = launch_connectivity(d_in, d_out, h->p.width, h->p.height, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "connectivity kernel launch");
    ++h->launches;
    return SLIC_OK;
}

slic_status slic_connectivity_components(slic_handle h, const int32_t *d_in, int32_t *d_out, void *stream) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (!d_in || !d_out) return fail(h, SLIC_ERR_INVALID, "NULL buffer");
    if (!h->ccl) return fail(h, SLIC_ERR_STATE, "the handle was not created with enforce_connectivity = 2");
    cudaError_t e = launch_connectivity_components(d_in, d_out, h->p.width, h->p.height, h->S * h->S / 4, h->ccl,
                                                   h->ccl_err, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "component connectivity launch");
    h->launches += 9;
    return SLIC_OK;
}

slic_status slic_status_check(slic_handle h) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    int flag = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, h->ccl_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag) e = cudaMemset(h->ccl_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    if (flag) return fail(h, SLIC_ERR_TIMEOUT, "a bounded device loop gave up");
    return SLIC_OK;
}

slic_status slic_launch_count(slic_handle h, long long *count) {
    if (!h || !count) return fail(h, SLIC_ERR_INVALID, "NULL argument");
    *count = h->launches;
    return SLIC_OK;
}

slic_status slic_profile_enable(slic_handle h, int enable) {
    if (!h) return fail(nullptr, SLIC_ERR_INVALID, "NULL handle");
    if (enable && !h->profiling) h->ev_used = 0;
    h->profiling = enable != 0;
    return SLIC_OK;
}

slic_status slic_profile_read(slic_handle h, double *assign_ms, long long *assign_launches) {
    if (!h || !assign_ms || !assign_launches) return fail(h, SLIC_ERR_INVALID, "NULL argument");
    double total = 0.0;
    for (size_t i = 0; i < h->ev_used; ++i) {
        cudaError_t e = cudaEventSynchronize(h->events[i].second);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->events[i].first, h->events[i].second);
        if (e != cudaSuccess) return cuda_fail(h, e, "profile event");
        total += ms;
    }
    *assign_ms = total;
    *assign_launches = (long long)h->ev_used;
    return SLIC_OK;
}

slic_status slic_fault_inject(int kind, long long value) {
    if (value < 0) return fail(nullptr, SLIC_ERR_INVALID, "fault injection value must be >= 0");
    static std::mutex mu;
    static unsigned steps = 0;
    static int abort_copies = 0;
    std::lock_guard<std::mutex> lk(mu);
    switch (kind) {
    case SLIC_FAULT_ALLOC:
        g_fail_allocs.store(value);
        return SLIC_OK;
    case SLIC_FAULT_WALK_LIMIT:
        if (value > (long long)ccl_default_steps()) return fail(nullptr, SLIC_ERR_INVALID, "walk limit above the default");
        steps = (unsigned)value;
        break;
    case SLIC_FAULT_ABORT_COPIES:
        abort_copies = value != 0;
        break;
    default:
        return fail(nullptr, SLIC_ERR_INVALID, "unknown fault kind");
    }
    const cudaError_t e = set_fault_words(steps ? steps : ccl_default_steps(), abort_copies);
    if (e != cudaSuccess) return fail(nullptr, SLIC_ERR_CUDA, std::string("fault words: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

const char *slic_last_error(slic_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free segmentation (slic_segment_noalloc)
//
// For callers that must not allocate device memory at all: code that runs
// while a stream is being captured into a CUDA graph (where cudaMalloc is not
// permitted), processes whose device memory is owned by another allocator
// under a fixed budget, and latency-critical loops that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree. The scratch lives
// in one file-scope device array that every GPU which loads this library
// holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
// The first 256 bytes are a control block at a fixed place: the timeout flag
// of component connectivity (bit 1), read and cleared by
// slic_noalloc_status_check. Device memory of a module starts zeroed.
constexpr size_t kStaticCtrlBytes = 256;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// With the device current: the sRGB table and the kernels' shared-memory
// limit (once per device), and the device address of the static scratch,
// taken afresh on every call (the symbol itself is only a host-side stand-in).
slic_status static_setup(int dev, size_t smem, unsigned char **addr) {
    cudaError_t e = ensure_lut(dev);
    if (e == cudaSuccess) e = ensure_smem(dev, smem);
    if (e != cudaSuccess) return fail(nullptr, SLIC_ERR_CUDA, std::string("set-up: ") + cudaGetErrorString(e));
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
        return fail(nullptr, SLIC_ERR_CUDA,
                    std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
    *addr = static_cast<unsigned char *>(p);
    return SLIC_OK;
}

}  // namespace

extern "C" slic_status slic_segment_noalloc(const slic_params *params, const uint8_t *d_image, int32_t *d_labels,
                                            float *d_centres, void *stream) {
    if (!params || !d_image || !d_labels || !d_centres) return fail(nullptr, SLIC_ERR_INVALID, "NULL argument");
    const slic_params &p = *params;
    if (p.width <= 0 || p.height <= 0 || p.width > (1 << 20) || p.height > (1 << 20) ||
        (long long)p.width * p.height >= (1LL << 31))
        return fail(nullptr, SLIC_ERR_INVALID, "width and height must be in [1, 2^20] with width*height < 2^31");
    if (p.S < 0 || (p.S == 0 && p.K <= 0)) return fail(nullptr, SLIC_ERR_INVALID, "need S > 0 or K > 0");
    if (!(p.m >= 0.0f) || !std::isfinite(p.m)) return fail(nullptr, SLIC_ERR_INVALID, "m must be finite and >= 0");
    if (p.iterations < 0) return fail(nullptr, SLIC_ERR_INVALID, "iterations must be >= 0");
    if (p.color_space < 0 || p.color_space > 2) return fail(nullptr, SLIC_ERR_INVALID, "unknown color_space");
    if (p.in_channels != 3 && p.in_channels != 4) return fail(nullptr, SLIC_ERR_INVALID, "in_channels must be 3 or 4");
    if (p.enforce_connectivity < 0 || p.enforce_connectivity > 2)
        return fail(nullptr, SLIC_ERR_INVALID, "enforce_connectivity must be 0, 1 or 2");
    if (p.perturb_seeds != 0 && p.perturb_seeds != 1)
        return fail(nullptr, SLIC_ERR_INVALID, "perturb_seeds must be 0 or 1");
    if (!(p.convergence >= 0.0f) || !std::isfinite(p.convergence))
        return fail(nullptr, SLIC_ERR_INVALID, "convergence must be finite and >= 0");
    int S = p.S;
    if (S == 0) {
        S = (int)std::lround(std::sqrt((double)p.width * (double)p.height / (double)p.K));
        if (S < 1) S = 1;
    }
    const int ns_c = (p.width + S - 1) / S, ns_r = (p.height + S - 1) / S;
    const long long K = (long long)ns_c * ns_r;
    const int P = (p.width + 3) & ~3;
    // Scratch layout: control block | features [3][H][P] f32 | sums [K][6] i64
    // | labels [H][W] i32 | stopping-test state | component scratch (mode 2).
    const size_t feat_b = align256(sizeof(float) * 3 * (size_t)p.height * P);
    const size_t acc_b = align256(sizeof(long long) * 6 * (size_t)K);
    const size_t lbl_b = align256(sizeof(int32_t) * (size_t)p.width * p.height);
    const size_t cs_b = align256(sizeof(ConvState));
    const size_t ccl_b =
        p.enforce_connectivity == 2 ? align256(sizeof(int) * ccl_scratch_ints((long long)p.width * p.height)) : 0;
    const size_t need = kStaticCtrlBytes + feat_b + acc_b + lbl_b + cs_b + ccl_b;
    if (need > kStaticScratchBytes)
        return fail(nullptr, SLIC_ERR_INVALID,
                    "image too large for the static scratch: needs " + std::to_string(need) +
                        " bytes, the limit is " + std::to_string(kStaticScratchBytes) + " (32 MiB)");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, SLIC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    const int win = assign_max_window(S, ns_c, ns_r);
    unsigned char *ctrl = nullptr;
    slic_status st = static_setup(dev, assign_smem_bytes(win, true), &ctrl);
    if (st != SLIC_OK) return st;
    unsigned char *const base = ctrl + kStaticCtrlBytes;

    FrameArgs a{};
    a.conv = make_conv(p.color_space);
    a.rgb = d_image;
    a.feat = reinterpret_cast<float *>(base);
    a.centres = d_centres;
    a.centres_out = d_centres;
    a.acc = reinterpret_cast<long long *>(base + feat_b);
    a.labels = d_labels;
    a.W = p.width;
    a.H = p.height;
    a.P = P;
    a.C = p.in_channels;
    a.S = S;
    a.ns_c = ns_c;
    a.ns_r = ns_r;
    a.w = p.m / (float)S;
    a.win_max = win;
    a.direct_acc = assign_direct_acc(win) ? 1 : 0;
    a.rgb_vec = ((p.width & 3) == 0 && ((uintptr_t)d_image & 15) == 0) ? 1 : 0;
    a.labels_vec = ((p.width & 3) == 0 && ((uintptr_t)d_labels & 15) == 0) ? 1 : 0;
    a.fix_scale = p.color_space == SLIC_RGB ? 1.0f : kFixScaleFrac;
    a.s_mul = S <= 2048 ? (unsigned)((0x100000000ULL + (unsigned)S - 1) / (unsigned)S) : 0u;
    a.tiles_x = (p.width + kTileW - 1) / kTileW;
    a.perturb = p.perturb_seeds;
    a.cstate = reinterpret_cast<ConvState *>(base + feat_b + acc_b + lbl_b);
    a.conv_eps = p.convergence;
    int32_t *lbl_tmp = reinterpret_cast<int32_t *>(base + feat_b + acc_b);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = assign_smem_bytes(win, true);

    // Same stage order as slic_segment; the initialisation kernel zeroes the
    // sums left in the shared array by the previous call.
    e = launch_init_from_rgb(a, s);
    for (int pass = 0; e == cudaSuccess && pass <= p.iterations; ++pass) {
        if (pass > 0)
            e = launch_update(a.acc, d_centres, d_centres, (int)K, 1.0f / a.fix_scale, a.cstate, a.conv_eps, pass, s);
        if (e == cudaSuccess) e = launch_assign(a, pass == 0, pass == p.iterations, false, smem, s);
    }
    if (e == cudaSuccess && p.enforce_connectivity == 1) {
        e = launch_connectivity(d_labels, lbl_tmp, p.width, p.height, s);
        if (e == cudaSuccess) e = launch_connectivity(lbl_tmp, d_labels, p.width, p.height, s);
    } else if (e == cudaSuccess && p.enforce_connectivity == 2) {
        e = launch_connectivity_components(d_labels, d_labels, p.width, p.height, S * S / 4,
                                           reinterpret_cast<int *>(base + feat_b + acc_b + lbl_b + cs_b),
                                           reinterpret_cast<int *>(ctrl), s);
    }
    if (e != cudaSuccess) return fail(nullptr, SLIC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

extern "C" slic_status slic_noalloc_status_check(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    void *p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_static_scratch);
    int flag = 0;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag) e = cudaMemset(p, 0, sizeof(int));
    if (e != cudaSuccess) return fail(nullptr, SLIC_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (flag) return fail(nullptr, SLIC_ERR_TIMEOUT, "a bounded device loop of the allocation-free path gave up");
    return SLIC_OK;
}
