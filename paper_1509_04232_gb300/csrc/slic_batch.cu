// Batched C ABI of libslicgb.so (declared and documented in include/slic.h):
// many frames of uneven resolution, superpixel size and compactness
// segmented by one set of launches per pass (a persistent assignment kernel
// loops over the tiles of all frames), plus the autotuner of its launch
// shape.
#include "slic.h"
#include "slic_internal.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <tuple>
#include <vector>

using namespace slicgb;

struct slic_batch_ctx {
    int n = 0;
    int iterations = 0;
    int connectivity = 0;
    int device = 0;
    int sms = 0;
    std::vector<slic_params> params;
    std::vector<FrameArgs> frames;    // host copy of the descriptor table
    // Device tables read by the kernels: the frame descriptors, the
    // component-connectivity frames and the image pointers of the warm
    // start, in two copies (a rebind fills the other one, stream-ordered,
    // from its own page-locked staging copy); d_* point into the current one.
    unsigned char *tables = nullptr, *staging = nullptr;
    size_t tbl_bytes = 0, tbl_ccl = 0, tbl_img = 0;
    int tbl_cur = 0;
    cudaEvent_t staged[2] = {nullptr, nullptr};  // the staging copy's last upload
    FrameArgs *d_frames = nullptr;
    unsigned char *scratch = nullptr; // features, sums, connectivity labels of all frames
    int *ccl = nullptr;               // component connectivity (mode 2): scratch over all frames' pixels
    CclFrame *d_ccl = nullptr;
    std::vector<CclFrame> ccl_frames;
    int ccl_tiles_total = 0;          // 32x32 tiles of all frames (component connectivity)
    std::vector<const uint8_t *> images;
    bool any_conv = false;            // some frame has a stopping threshold
    int total_tiles = 0, total_centres = 0, total_rows = 0, max_w = 0, win_max = 0;
    int total_tiles64 = 0, win_max64 = 0;  // the same for 32x64 tiles
    int total_chunks = 0;    // update chunks of all frames (fused passes)
    bool fused = false;      // the passes before the last in one cooperative launch
    // Groups: the frames run as `groups` runs of consecutive frames (split
    // by pixel count), each enqueued on its own stream (the caller's for the
    // first, internal ones for the others, forked from and joined back to
    // the caller's stream by events), so one group's pass boundaries overlap
    // another's passes. Each group has a frame table of its own in the tables
    // block, its bases counted from its first frame.
    int groups = 1;
    std::vector<int> group_first;              // groups + 1 frame indices
    size_t tbl_grp = 0;                        // offset of the group tables in the tables block
    const FrameArgs *d_group_frames = nullptr; // (in the current tables block)
    cudaStream_t gstream[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
    int total_units = 0;  // work units of the fused connectivity kernel
    long long total_pixels = 0;
    bool same = true;        // every frame's S a multiple of 4 (4-pixel groups share a cell)
    bool same8 = true;       // every frame's S a multiple of 8 (two row groups share a cell row)
    bool pipe = false;       // passes after the first use the pipelined kernel
    bool buffers_set = false;
    size_t smem = 0;
    int occupancy = 0;       // resident CTAs per SM of the first-pass kernel
    int max_ring = 0;
    int *d_err = nullptr;    // device flag: a bounded wait timed out
    int ctas_per_sm = 0;     // 0: as many as fit
    int stages = 4;          // TMA pipeline stages of the pipelined kernel (3..4)
    int rows = 1;            // row groups per warp of the pipelined kernel (1, or 2 when same8)
    int tile_h = 32;         // tile rows of the pipelined kernel (32, or 64 with rows = 2)
    long long launches = 0;
    // learned warm start (slic_batch_set_warmstart): the network, its labels
    // [n][H][W] and the device table of the frames' image pointers
    slic_net net = nullptr;
    int32_t *net_labels = nullptr;
    const uint8_t *const *d_img_table = nullptr;  // (in the tables block)
    int net_C = 3;
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    size_t ev_used = 0;
    std::string err;
};

namespace {

thread_local std::string g_batch_error = "no error";

slic_status bfail(slic_batch_ctx *b, slic_status st, const std::string &msg) {
    if (b)
        b->err = msg;
    else
        g_batch_error = msg;
    return st;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

// cuTensorMapEncodeTiled from the driver, found once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 slicgb::tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

namespace {

// Tensor maps of one frame for the pipelined assignment: the features as a
// [3][H][P] f32 tensor copied in 32x32x3 (or 32x64x3) boxes, and the padded
// centre table as a [ns_r+2][(ns_c+2)*kCtabRec] f32 tensor copied in
// box_h x box_w*kCtabRec (or box_h64 x box_w*kCtabRec) boxes (the innermost
// coordinate of a copy, (wx0+1)*kCtabRec floats, is a multiple of 16 bytes).
bool encode_maps(FrameArgs &a) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || a.box_w * kCtabRec > 256 || a.box_h64 > 256) return false;
    const cuuint64_t fdim[3] = {(cuuint64_t)a.P, (cuuint64_t)a.H, 3};
    const cuuint64_t fstride[2] = {(cuuint64_t)a.P * 4, (cuuint64_t)a.P * a.H * 4};
    const cuuint32_t fbox[3] = {(cuuint32_t)kTileW, (cuuint32_t)kTileH, 3};
    const cuuint32_t ones[3] = {1, 1, 1};
    if (enc(&a.feat_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.feat, fdim, fstride, fbox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t cdim[2] = {(cuuint64_t)(a.ns_c + 2) * kCtabRec, (cuuint64_t)(a.ns_r + 2)};
    const cuuint64_t cstride[1] = {(cuuint64_t)(a.ns_c + 2) * kCtabRec * 4};
    const cuuint32_t cbox[2] = {(cuuint32_t)a.box_w * kCtabRec, (cuuint32_t)a.box_h};
    if (enc(&a.ctab_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, a.ctab, cdim, cstride, cbox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    // 32x64 tiles: a box twice as high, and the taller window of centres
    const cuuint32_t fbox64[3] = {(cuuint32_t)kTileW, (cuuint32_t)(2 * kTileH), 3};
    const cuuint32_t cbox64[2] = {(cuuint32_t)a.box_w * kCtabRec, (cuuint32_t)a.box_h64};
    return enc(&a.feat_map64, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.feat, fdim, fstride, fbox64, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
           enc(&a.ctab_map64, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, a.ctab, cdim, cstride, cbox64, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool valid_params(const slic_params &p, std::string &why) {
    if (p.width <= 0 || p.height <= 0 || p.width > (1 << 20) || p.height > (1 << 20) ||
        (long long)p.width * p.height >= (1LL << 31)) {
        why = "width and height must be in [1, 2^20] with width*height < 2^31";
        return false;
    }
    if (p.S < 0 || (p.S == 0 && p.K <= 0)) { why = "need S > 0 or K > 0"; return false; }
    if (!(p.m >= 0.0f) || !std::isfinite(p.m)) { why = "m must be finite and >= 0"; return false; }
    if (p.iterations < 0) { why = "iterations must be >= 0"; return false; }
    if (p.color_space < 0 || p.color_space > 2) { why = "unknown color_space"; return false; }
    if (p.in_channels != 3 && p.in_channels != 4) { why = "in_channels must be 3 or 4"; return false; }
    if (p.enforce_connectivity < 0 || p.enforce_connectivity > 2) {
        why = "enforce_connectivity must be 0, 1 or 2";
        return false;
    }
    if (p.perturb_seeds != 0 && p.perturb_seeds != 1) { why = "perturb_seeds must be 0 or 1"; return false; }
    if (!(p.convergence >= 0.0f) || !std::isfinite(p.convergence)) {
        why = "convergence must be finite and >= 0";
        return false;
    }
    return true;
}

// Persistent grids: CTAs per SM requested (or all that fit), capped by the
// occupancy of the kernel being launched.
int grid_for(const slic_batch_ctx *b, int occ) {
    const int per_sm = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, occ) : occ;
    return std::max(1, per_sm) * b->sms;
}

int pipe_occ(const slic_batch_ctx *b, int stages, int rows, int tile_h) {
    return std::max(1, assign_pipe_occupancy(b->same, tile_h == 64 ? b->win_max64 : b->win_max, stages, rows, tile_h));
}

// Whether a launch shape of the pipelined kernel fits (shared memory) and is
// allowed for the batch.
bool shape_fits(const slic_batch_ctx *b, int stages, int rows, int tile_h) {
    if (!b->pipe) return rows == 1 && tile_h == 32;
    if ((rows == 2 || tile_h == 64) && !b->same8) return false;
    if (tile_h == 64 && rows != 2) return false;
    return assign_pipe_occupancy(b->same, tile_h == 64 ? b->win_max64 : b->win_max, stages, rows, tile_h) > 0;
}

std::string tune_key(const slic_batch_ctx *b) {
    cudaDeviceProp prop;
    std::string gpu = cudaGetDeviceProperties(&prop, b->device) == cudaSuccess ? prop.name : "unknown";
    std::set<std::tuple<int, int, int>> shapes;
    for (const FrameArgs &f : b->frames) shapes.insert(std::make_tuple(f.W, f.H, f.S));
    std::string key = gpu + "|frames=" + std::to_string(b->n) + "|it=" + std::to_string(b->iterations);
    for (const auto &s : shapes)
        key += "|" + std::to_string(std::get<0>(s)) + "x" + std::to_string(std::get<1>(s)) + "s" +
               std::to_string(std::get<2>(s));
    for (char &c : key)
        if (c == '"' || c == '\\' || c == '\n') c = '_';
    return key;
}

// Cache lines: {"key": "<key>", "ctas_per_sm": <int>, "stages": <int>, "rows": <int>, "tile_h": <int>,
// "fused": <0|1>, "groups": <int>, "ms": <float>}
bool cache_lookup(const char *path, const std::string &key, int *ctas, int *stages, int *rows, int *tile_h,
                  int *fused, int *groups) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[4096];
    bool found = false;
    const std::string needle = "\"key\": \"" + key + "\"";
    while (std::fgets(line, sizeof line, f)) {
        if (std::strstr(line, needle.c_str())) {
            const char *q = std::strstr(line, "\"ctas_per_sm\":");
            const char *r = std::strstr(line, "\"stages\":");
            const char *o = std::strstr(line, "\"rows\":");
            const char *t = std::strstr(line, "\"tile_h\":");
            const char *z = std::strstr(line, "\"fused\":");
            const char *gp = std::strstr(line, "\"groups\":");
            int v = 0, w = 0, u = 0, h = 0, fz = -1, gn = 0;
            if (q && r && o && t && z && gp && std::sscanf(q + 14, "%d", &v) == 1 &&
                std::sscanf(r + 9, "%d", &w) == 1 && std::sscanf(o + 7, "%d", &u) == 1 &&
                std::sscanf(t + 9, "%d", &h) == 1 && std::sscanf(z + 8, "%d", &fz) == 1 &&
                std::sscanf(gp + 9, "%d", &gn) == 1 && v > 0 && w >= 3 && w <= 4 && (u == 1 || u == 2) &&
                (h == 32 || h == 64) && (fz == 0 || fz == 1) && gn >= 1 && gn <= 4) {
                *groups = gn;
                *ctas = v;
                *stages = w;
                *rows = u;
                *tile_h = h;
                *fused = fz;
                found = true;
            }
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, int ctas, int stages, int rows, int tile_h, int fused,
                 int groups, float ms) {
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"ctas_per_sm\": %d, \"stages\": %d, \"rows\": %d, \"tile_h\": %d, "
                 "\"fused\": %d, \"groups\": %d, \"ms\": %.4f}\n",
                 key.c_str(), ctas, stages, rows, tile_h, fused, groups, ms);
    std::fclose(f);
}

// The frames' buffers into the host tables (frame descriptors,
// component-connectivity frames).
void bind_frames(slic_batch_ctx *b, const uint8_t *const *d_images, int32_t *const *d_labels, float *const *d_centres,
                 const float *const *d_init) {
    for (int f = 0; f < b->n; ++f) {
        FrameArgs &a = b->frames[f];
        b->images[f] = d_images[f];
        a.rgb = d_images[f];
        a.labels = d_labels[f];
        a.centres = d_centres[f];
        a.centres_out = d_centres[f];
        a.init = d_init ? d_init[f] : nullptr;
        a.rgb_vec = ((a.W & 3) == 0 && ((uintptr_t)a.rgb & 15) == 0) ? 1 : 0;
        a.labels_vec = ((a.W & 3) == 0 && ((uintptr_t)a.labels & 15) == 0) ? 1 : 0;
        // The pipelined last pass writes lbl_tmp when the fused connectivity
        // kernel follows (it reads lbl_tmp and writes the labels).
        const bool fused = b->pipe && b->connectivity == 1;
        a.assign_out = fused ? a.lbl_tmp : a.labels;
        a.assign_vec = fused ? ((a.W & 3) == 0 ? 1 : 0) : a.labels_vec;
    }
    if (b->connectivity == 2) {
        b->ccl_frames.assign(b->n, CclFrame{});
        int base = 0, tile_base = 0;
        for (int f = 0; f < b->n; ++f) {
            const FrameArgs &a = b->frames[f];
            b->ccl_frames[f] = CclFrame{a.labels, a.labels, a.W, a.S * a.S / 4, base, a.H, tile_base};
            base += a.W * a.H;
            tile_base += ccl_tiles(a.W, a.H);
        }
        b->ccl_tiles_total = tile_base;
    }
}

// Upload the host tables into device copy k, ordered on stream s (the
// staging copy k is reused only after its previous upload completed), and
// make it the current one; then the sentinel ring of the centre tables.
cudaError_t upload_tables(slic_batch_ctx *b, int k, cudaStream_t s) {
    cudaError_t e = cudaEventSynchronize(b->staged[k]);
    if (e != cudaSuccess) return e;
    unsigned char *h = b->staging + (size_t)k * b->tbl_bytes, *d = b->tables + (size_t)k * b->tbl_bytes;
    std::memcpy(h, b->frames.data(), sizeof(FrameArgs) * b->n);
    if (b->connectivity == 2) std::memcpy(h + b->tbl_ccl, b->ccl_frames.data(), sizeof(CclFrame) * b->n);
    std::memcpy(h + b->tbl_img, b->images.data(), sizeof(const uint8_t *) * b->n);
    // group tables: the frames again, each group's bases counted from its
    // first frame (its kernels index tiles, centres, rows, connectivity
    // units and update chunks from 0)
    FrameArgs *gt = reinterpret_cast<FrameArgs *>(h + b->tbl_grp);
    for (int g = 0; g < b->groups; ++g) {
        const FrameArgs &a0 = b->frames[b->group_first[g]];
        for (int f = b->group_first[g]; f < b->group_first[g + 1]; ++f) {
            FrameArgs a = b->frames[f];
            a.tile_base -= a0.tile_base;
            a.tile_base64 -= a0.tile_base64;
            a.centre_base -= a0.centre_base;
            a.row_base -= a0.row_base;
            a.strip_base -= a0.strip_base;
            a.chunk_base -= a0.chunk_base;
            gt[f] = a;
        }
    }
    e = cudaMemcpyAsync(d, h, b->tbl_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->staged[k], s);
    if (e != cudaSuccess) return e;
    b->tbl_cur = k;
    b->d_frames = reinterpret_cast<FrameArgs *>(d);
    b->d_ccl = reinterpret_cast<CclFrame *>(d + b->tbl_ccl);
    b->d_img_table = reinterpret_cast<const uint8_t *const *>(d + b->tbl_img);
    b->d_group_frames = reinterpret_cast<const FrameArgs *>(d + b->tbl_grp);
    return launch_fill_ring(b->d_frames, b->n, b->max_ring, s);
}

}  // namespace

extern "C" {

slic_status slic_batch_create(const slic_params *params, int n_frames, slic_batch *out) {
    if (!params || !out || n_frames <= 0) return bfail(nullptr, SLIC_ERR_INVALID, "need params, n_frames > 0 and out");
    *out = nullptr;
    std::string why;
    for (int f = 0; f < n_frames; ++f) {
        if (!valid_params(params[f], why)) return bfail(nullptr, SLIC_ERR_INVALID, "frame " + std::to_string(f) + ": " + why);
        if (params[f].iterations != params[0].iterations ||
            params[f].enforce_connectivity != params[0].enforce_connectivity)
            return bfail(nullptr, SLIC_ERR_INVALID, "all frames of a batch need the same iterations and connectivity");
    }
    slic_batch_ctx *b = new (std::nothrow) slic_batch_ctx;
    if (!b) return bfail(nullptr, SLIC_ERR_NOMEM, "host allocation failed");
    b->n = n_frames;
    b->iterations = params[0].iterations;
    b->connectivity = params[0].enforce_connectivity;
    b->params.assign(params, params + n_frames);
    b->frames.resize(n_frames);

    // Geometry, bases and the scratch layout.
    size_t bytes = 0;
    std::vector<size_t> off_feat(n_frames), off_acc(n_frames), off_lbl(n_frames), off_ctab(n_frames),
        off_cs(n_frames);
    long long tiles = 0, tiles64 = 0, centres = 0, rows = 0;
    for (int f = 0; f < n_frames; ++f) {
        const slic_params &p = params[f];
        FrameArgs &a = b->frames[f];
        std::memset(&a, 0, sizeof a);
        int S = p.S;
        if (S == 0) {
            S = (int)std::lround(std::sqrt((double)p.width * (double)p.height / (double)p.K));
            if (S < 1) S = 1;
        }
        a.conv = conv_consts(p.color_space);
        a.W = p.width;
        a.H = p.height;
        a.P = (p.width + 3) & ~3;
        a.C = p.in_channels;
        a.S = S;
        a.ns_c = (p.width + S - 1) / S;
        a.ns_r = (p.height + S - 1) / S;
        a.w = p.m / (float)S;
        a.fix_scale = p.color_space == SLIC_RGB ? 1.0f : kFixScaleFrac;
        a.s_mul = S <= 2048 ? (unsigned)((0x100000000ULL + (unsigned)S - 1) / (unsigned)S) : 0u;
        a.tiles_x = (p.width + kTileW - 1) / kTileW;
        a.perturb = p.perturb_seeds;
        a.conv_eps = p.convergence;
        b->any_conv = b->any_conv || p.convergence > 0.0f;
        a.tile_base = (int)tiles;
        a.centre_base = (int)centres;
        a.row_base = (int)rows;
        a.tile_base64 = (int)tiles64;
        a.n_tiles = a.tiles_x * ((p.height + kTileH - 1) / kTileH);
        a.n_tiles64 = a.tiles_x * ((p.height + 2 * kTileH - 1) / (2 * kTileH));
        a.n_chunks = (a.ns_c * a.ns_r + kUpdateChunk - 1) / kUpdateChunk;
        tiles += a.n_tiles;
        tiles64 += a.n_tiles64;
        centres += (long long)a.ns_c * a.ns_r;
        rows += p.height;
        if (tiles >= (1LL << 31) || centres >= (1LL << 31) || rows >= (1LL << 31)) {
            delete b;
            return bfail(nullptr, SLIC_ERR_INVALID, "batch too large (tiles, centres or rows exceed 2^31)");
        }
        b->win_max = std::max(b->win_max, assign_max_window(S, a.ns_c, a.ns_r));
        b->win_max64 = std::max(b->win_max64, assign_max_window(S, a.ns_c, a.ns_r, 2 * kTileH));
        {
            const int span = (kTileW - 1) / S + 2, spanh = (kTileH - 1) / S + 2, spanh64 = (2 * kTileH - 1) / S + 2;
            a.box_w = std::min(span, a.ns_c) + 2;
            a.box_h = std::min(spanh, a.ns_r) + 2;
            a.box_h64 = std::min(spanh64, a.ns_r) + 2;
        }
        b->max_w = std::max(b->max_w, p.width);
        a.strip_base = b->total_units;
        b->total_units += connectivity2_units(p.width, p.height, &a.strips_x);
        b->same = b->same && (S % kPPT) == 0;
        b->same8 = b->same8 && (S % 8) == 0;
        b->total_pixels += (long long)p.width * p.height;
        off_feat[f] = bytes;
        bytes += align256(sizeof(float) * 3 * (size_t)p.height * a.P);
        off_acc[f] = bytes;
        bytes += align256(sizeof(long long) * 6 * (size_t)a.ns_c * a.ns_r);
        off_lbl[f] = bytes;
        bytes += align256(sizeof(int32_t) * (size_t)p.width * p.height);
        off_ctab[f] = bytes;
        bytes += align256(sizeof(float) * kCtabRec * (size_t)(a.ns_c + 2) * (a.ns_r + 2));
        off_cs[f] = bytes;
        bytes += align256(sizeof(ConvState));
        b->max_ring = std::max(b->max_ring, 2 * (a.ns_c + 2) + 2 * a.ns_r);
    }
    const size_t off_err = bytes;
    bytes += 256;
    // component connectivity: one scratch over all frames' pixels and the table
    size_t off_ccl = 0;
    if (b->connectivity == 2) {
        if (b->total_pixels >= (1LL << 31)) {
            delete b;
            return bfail(nullptr, SLIC_ERR_INVALID, "component connectivity needs fewer than 2^31 pixels per batch");
        }
        off_ccl = bytes;
        bytes += align256(sizeof(int) * ccl_scratch_ints(b->total_pixels));
    }
    b->tbl_ccl = align256(sizeof(FrameArgs) * (size_t)n_frames);
    b->tbl_img = b->tbl_ccl + align256(sizeof(CclFrame) * (size_t)n_frames);
    b->tbl_grp = b->tbl_img + align256(sizeof(const uint8_t *) * (size_t)n_frames);
    b->tbl_bytes = b->tbl_grp + align256(sizeof(FrameArgs) * (size_t)n_frames);
    b->group_first = {0, n_frames};
    b->total_tiles = (int)tiles;
    b->total_tiles64 = (int)tiles64;
    {
        long long chunks = 0;  // the batch's update chunks (fused passes), frame after frame
        for (FrameArgs &a : b->frames) {
            a.chunk_base = (int)chunks;
            chunks += a.n_chunks;
        }
        b->total_chunks = (int)chunks;  // (< total_centres, checked above)
    }
    b->total_centres = (int)centres;
    b->total_rows = (int)rows;
    for (FrameArgs &a : b->frames) {
        a.win_max = b->win_max;
        a.direct_acc = assign_direct_acc(b->win_max) ? 1 : 0;
    }
    b->smem = assign_smem_bytes(b->win_max, true);

    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = device_setup(b->device, b->smem);
    if (e != cudaSuccess) {
        delete b;
        return bfail(nullptr, SLIC_ERR_CUDA, std::string("CUDA set-up: ") + cudaGetErrorString(e));
    }
    // The pipelined kernel needs private sums and its shared memory within
    // the opt-in limit (at least with three stages).
    b->same8 = b->same8 && b->same;
    b->pipe = !assign_direct_acc(b->win_max) && assign_pipe_occupancy(b->same, b->win_max, 3, 1) > 0;
    if (b->pipe && assign_pipe_occupancy(b->same, b->win_max, 4, 1) == 0) b->stages = 3;
    b->occupancy = std::max(1, assign_batch_occupancy(b->same, b->smem));
    if (dev_alloc(&b->scratch, bytes) != cudaSuccess || dev_alloc(&b->tables, 2 * b->tbl_bytes) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&b->staging), 2 * b->tbl_bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->scratch);
        cudaFree(b->tables);
        delete b;
        return bfail(nullptr, SLIC_ERR_NOMEM, "allocation of " + std::to_string(bytes) + " device bytes failed");
    }
    if (cudaEventCreateWithFlags(&b->staged[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->staged[1], cudaEventDisableTiming) != cudaSuccess) {
        slic_batch_destroy(b);
        return bfail(nullptr, SLIC_ERR_CUDA, "cudaEventCreate failed");
    }
    b->images.assign(n_frames, nullptr);
    b->d_frames = reinterpret_cast<FrameArgs *>(b->tables);
    b->d_ccl = reinterpret_cast<CclFrame *>(b->tables + b->tbl_ccl);
    for (int f = 0; f < n_frames; ++f) {
        FrameArgs &a = b->frames[f];
        a.feat = reinterpret_cast<float *>(b->scratch + off_feat[f]);
        a.acc = reinterpret_cast<long long *>(b->scratch + off_acc[f]);
        a.lbl_tmp = reinterpret_cast<int32_t *>(b->scratch + off_lbl[f]);
        a.ctab = reinterpret_cast<float *>(b->scratch + off_ctab[f]);
        a.cstate = reinterpret_cast<ConvState *>(b->scratch + off_cs[f]);
        if (b->pipe && !encode_maps(a)) b->pipe = false;  // then every pass uses k_assign_batch
    }
    b->d_err = reinterpret_cast<int *>(b->scratch + off_err);
    if (b->connectivity == 2) b->ccl = reinterpret_cast<int *>(b->scratch + off_ccl);
    if (cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess) {
        slic_batch_destroy(b);
        return bfail(nullptr, SLIC_ERR_CUDA, "clearing the error flag failed");
    }
    *out = b;
    return SLIC_OK;
}

slic_status slic_batch_destroy(slic_batch b) {
    if (!b) return SLIC_OK;
    cudaDeviceSynchronize();
    cudaFree(b->scratch);
    cudaFree(b->tables);
    cudaFreeHost(b->staging);
    for (cudaEvent_t ev : b->staged)
        if (ev) cudaEventDestroy(ev);
    for (int g = 0; g < 3; ++g) {
        if (b->gstream[g]) cudaStreamDestroy(b->gstream[g]);
        if (b->ev_join[g]) cudaEventDestroy(b->ev_join[g]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    cudaFree(b->net_labels);
    for (auto &ev : b->events) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    delete b;
    return SLIC_OK;
}

slic_status slic_batch_set_buffers(slic_batch b, const uint8_t *const *d_images, int32_t *const *d_labels,
                                   float *const *d_centres, const float *const *d_init) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (!d_images || !d_labels || !d_centres) return bfail(b, SLIC_ERR_INVALID, "NULL pointer array");
    for (int f = 0; f < b->n; ++f)
        if (!d_images[f] || !d_labels[f] || !d_centres[f])
            return bfail(b, SLIC_ERR_INVALID, "NULL buffer for frame " + std::to_string(f));
    // Synchronous: the tables must not change under queued work.
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        bind_frames(b, d_images, d_labels, d_centres, d_init);
        e = upload_tables(b, b->tbl_cur, nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("frame table upload: ") + cudaGetErrorString(e));
    b->buffers_set = true;
    return SLIC_OK;
}

slic_status slic_batch_rebind(slic_batch b, const uint8_t *const *d_images, int32_t *const *d_labels,
                              float *const *d_centres, const float *const *d_init, void *stream) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (!b->buffers_set) return bfail(b, SLIC_ERR_STATE, "slic_batch_set_buffers has not been called");
    if (!d_images || !d_labels || !d_centres) return bfail(b, SLIC_ERR_INVALID, "NULL pointer array");
    for (int f = 0; f < b->n; ++f)
        if (!d_images[f] || !d_labels[f] || !d_centres[f])
            return bfail(b, SLIC_ERR_INVALID, "NULL buffer for frame " + std::to_string(f));
    bind_frames(b, d_images, d_labels, d_centres, d_init);
    const cudaError_t e = upload_tables(b, b->tbl_cur ^ 1, (cudaStream_t)stream);
    if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("frame table upload: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

}  // extern "C"

namespace {

// A run of consecutive frames as the kernels see it: its device frame table
// (bases counted from its first frame) and its totals.
struct Span {
    const FrameArgs *frames;
    int n, tiles, tiles64, centres, rows, units, chunks;
};

// Group g of the batch (g < 0: the whole batch, with its own table).
Span span_of(const slic_batch_ctx *b, int g) {
    if (g < 0)
        return Span{b->d_frames, b->n, b->total_tiles, b->total_tiles64, b->total_centres, b->total_rows,
                    b->total_units, b->total_chunks};
    const int f0 = b->group_first[g], f1 = b->group_first[g + 1];
    const FrameArgs &a = b->frames[f0];
    const bool end = f1 == b->n;
    const FrameArgs *z = end ? nullptr : &b->frames[f1];
    return Span{b->d_group_frames + f0, f1 - f0,
                (end ? b->total_tiles : z->tile_base) - a.tile_base,
                (end ? b->total_tiles64 : z->tile_base64) - a.tile_base64,
                (end ? b->total_centres : z->centre_base) - a.centre_base,
                (end ? b->total_rows : z->row_base) - a.row_base,
                (end ? b->total_units : z->strip_base) - a.strip_base,
                (end ? b->total_chunks : z->chunk_base) - a.chunk_base};
}

// Every stage of a segmentation of the span's frames, enqueued on s: the
// conversion pre-pass (pipelined kernel) or the first pass's conversion,
// the initialisation, the learned warm start (whole batch only), the passes
// and updates (fused or one launch each), connectivity. `whole`: the span
// is the whole batch (the warm start, component connectivity and the
// profiling events need it).
cudaError_t enqueue_span(slic_batch_ctx *b, const Span &sp, cudaStream_t s, bool whole, long long &n_launch,
                         std::string &why) {
    const int grid = grid_for(b, b->occupancy);
    const int grid_pipe = b->pipe ? grid_for(b, pipe_occ(b, b->stages, b->rows, b->tile_h)) : grid;
    const int pipe_per_sm = grid_pipe / std::max(1, b->sms);
    // With the pipelined kernel every pass reads features: a conversion
    // pre-pass writes them, and the first pass is pipelined as well.
    cudaError_t e = cudaSuccess;
    if (b->pipe) {
        e = launch_convert_batch(sp.frames, sp.n, sp.rows, b->max_w, s);
        ++n_launch;
    }
    if (e == cudaSuccess) e = launch_init_batch(sp.frames, sp.n, sp.centres, s);
    ++n_launch;
    const bool warm = whole && b->net != nullptr;
    if (warm) {
        // Learned warm start: the network's labels, their member sums (from
        // the features of the pre-pass) and one update without the stopping
        // test's bookkeeping (update 0) turn them into the initial centres.
        if (e == cudaSuccess && !b->pipe) {
            e = launch_convert_batch(sp.frames, sp.n, sp.rows, b->max_w, s);
            ++n_launch;
        }
        if (e == cudaSuccess &&
            net_forward_labels(b->net, b->n, nullptr, b->d_img_table, b->net_C, b->net_labels, s) != cudaSuccess) {
            why = std::string("network forward: ") + slic_net_last_error(b->net);
            return cudaErrorLaunchFailure;
        }
        if (e == cudaSuccess) e = launch_accumulate_labels_batch(sp.frames, sp.n, sp.rows, b->max_w, s);
        if (e == cudaSuccess) e = launch_update_batch(sp.frames, sp.n, sp.centres, 0, s);
        n_launch += 2;
    }
    // Event pair around one assignment launch when profiling.
    auto timed = [&](auto launch) -> cudaError_t {
        cudaEvent_t e1 = nullptr;
        if (b->profiling && whole) {
            if (b->ev_used == b->events.size()) {
                cudaEvent_t x, y;
                if (cudaEventCreate(&x) != cudaSuccess || cudaEventCreate(&y) != cudaSuccess)
                    return cudaErrorMemoryAllocation;
                b->events.emplace_back(x, y);
            }
            const cudaError_t r = record_profile_event(b->events[b->ev_used].first, s);
            if (r != cudaSuccess) return r;
            e1 = b->events[b->ev_used++].second;
        }
        cudaError_t r = launch();
        if (e1 && r == cudaSuccess) r = record_profile_event(e1, s);
        ++n_launch;
        return r;
    };
    const int tiles_th = b->tile_h == 64 ? sp.tiles64 : sp.tiles;
    const int win_th = b->tile_h == 64 ? b->win_max64 : b->win_max;
    auto last_or_pass = [&](int pass) {
        return [&, pass]() {
            return b->pipe ? launch_assign_pipe(sp.frames, sp.n, tiles_th, win_th, b->same, pass == b->iterations,
                                                b->stages, b->rows, b->tile_h, pipe_per_sm, grid_pipe, b->d_err,
                                                b->any_conv ? 1 : 0, s)
                           : launch_assign_batch(sp.frames, sp.n, sp.tiles, b->win_max, b->same, pass == 0 && !warm,
                                                 pass == b->iterations, b->smem, grid, s);
        };
    };
    if (e == cudaSuccess && b->pipe && b->fused && whole && b->iterations > 0) {
        // Passes 0 .. n-1 with updates 1 .. n in one cooperative launch
        // (per-frame phase counters order them), then the last pass.
        const int occ = std::max(1, assign_pipe_occupancy(b->same, win_th, b->stages, b->rows, b->tile_h, true));
        const int grid_multi = grid_for(b, occ);
        e = timed([&]() {
            return launch_assign_multi(sp.frames, sp.n, tiles_th, sp.chunks, win_th, b->same, b->iterations,
                                       b->stages, b->rows, b->tile_h, grid_multi / std::max(1, b->sms), grid_multi,
                                       b->d_err, b->any_conv ? 1 : 0, s);
        });
        if (e == cudaSuccess) e = timed(last_or_pass(b->iterations));
    } else {
        for (int pass = 0; e == cudaSuccess && pass <= b->iterations; ++pass) {
            if (pass > 0) {
                e = launch_update_batch(sp.frames, sp.n, sp.centres, pass, s);
                ++n_launch;
            }
            if (e == cudaSuccess) e = timed(last_or_pass(pass));
        }
    }
    if (e == cudaSuccess && b->connectivity == 2) {
        // component-based connectivity over all frames at once, in place on the labels
        e = launch_connectivity_components(b->d_ccl, b->ccl_frames[0], b->n, (int)b->total_pixels, b->ccl_tiles_total,
                                           b->ccl, b->d_err,
                                           s);
        n_launch += 9;
    } else if (e == cudaSuccess && b->connectivity) {
        if (b->pipe) {
            e = launch_connectivity2_batch(sp.frames, sp.n, sp.units, b->sms * 8, s);
            n_launch += 1;
        } else {
            e = launch_connectivity_batch(sp.frames, sp.n, sp.rows, b->max_w, 0, s);
            if (e == cudaSuccess) e = launch_connectivity_batch(sp.frames, sp.n, sp.rows, b->max_w, 1, s);
            n_launch += 2;
        }
    }
    return e;
}

}  // namespace

extern "C" {

// Groups run concurrently only on the plain pipelined path (the warm start,
// component connectivity and the per-launch timers take the whole batch at
// once).
static bool split_groups(const slic_batch_ctx *b) {
    return b->groups > 1 && b->pipe && !b->net && b->connectivity != 2 && !b->profiling;
}

slic_status slic_batch_segment(slic_batch b, void *stream) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (!b->buffers_set) return bfail(b, SLIC_ERR_STATE, "slic_batch_set_buffers has not been called");
    cudaStream_t s = (cudaStream_t)stream;
    long long n_launch = 0;
    std::string why;
    cudaError_t e = cudaSuccess;
    if (!split_groups(b)) {
        e = enqueue_span(b, span_of(b, -1), s, true, n_launch, why);
    } else {
        e = cudaEventRecord(b->ev_fork, s);
        for (int g = 1; g < b->groups && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(b->gstream[g - 1], b->ev_fork, 0);
        for (int g = 0; g < b->groups && e == cudaSuccess; ++g)
            e = enqueue_span(b, span_of(b, g), g == 0 ? s : b->gstream[g - 1], false, n_launch, why);
        for (int g = 1; g < b->groups && e == cudaSuccess; ++g) {
            e = cudaEventRecord(b->ev_join[g - 1], b->gstream[g - 1]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[g - 1], 0);
        }
    }
    if (e != cudaSuccess)
        return bfail(b, SLIC_ERR_CUDA, why.empty() ? std::string("kernel launch: ") + cudaGetErrorString(e) : why);
    b->launches += n_launch;
    return SLIC_OK;
}

namespace {
// Copies of equal direction for frames 0..n-1 (host[f], device[f], bytes[f];
// a NULL host pointer skips the frame), one cudaMemcpyAsync for each run of
// frames that lie back to back in both host and device memory.
cudaError_t copy_runs(int n, const std::vector<const void *> &src, const std::vector<void *> &dst,
                      const std::vector<size_t> &bytes, cudaMemcpyKind kind, cudaStream_t s) {
    int f = 0;
    while (f < n) {
        if (!src[f]) {
            ++f;
            continue;
        }
        size_t len = bytes[f];
        int g = f + 1;
        while (g < n && src[g] && static_cast<const char *>(src[g]) == static_cast<const char *>(src[f]) + len &&
               static_cast<char *>(dst[g]) == static_cast<char *>(dst[f]) + len) {
            len += bytes[g];
            ++g;
        }
        const cudaError_t e = cudaMemcpyAsync(dst[f], src[f], len, kind, s);
        if (e != cudaSuccess) return e;
        f = g;
    }
    return cudaSuccess;
}
}  // namespace

slic_status slic_batch_segment_host(slic_batch b, const uint8_t *const *host_images, int32_t *const *host_labels,
                                    float *const *host_centres, void *stream) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (!host_images) return bfail(b, SLIC_ERR_INVALID, "NULL host image array");
    if (!b->buffers_set) return bfail(b, SLIC_ERR_STATE, "slic_batch_set_buffers has not been called");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = b->n;
    for (int f = 0; f < n; ++f)
        if (!host_images[f]) return bfail(b, SLIC_ERR_INVALID, "NULL host image for frame " + std::to_string(f));
    // The copies of frames f0 .. f1-1: images in (pass 0), or labels
    // (pass 1) and centres (pass 2) out, on stream t.
    auto copy_frames = [&](int f0, int f1, int pass, cudaStream_t t) -> cudaError_t {
        const int m = f1 - f0;
        std::vector<const void *> src(m);
        std::vector<void *> dst(m);
        std::vector<size_t> len(m);
        if (pass == 1 && !host_labels) return cudaSuccess;
        if (pass == 2 && !host_centres) return cudaSuccess;
        for (int i = 0; i < m; ++i) {
            const FrameArgs &a = b->frames[f0 + i];
            if (pass == 0) {
                src[i] = host_images[f0 + i];
                dst[i] = const_cast<uint8_t *>(a.rgb);
                len[i] = (size_t)a.W * a.H * a.C;
            } else {
                src[i] = pass == 1 ? static_cast<const void *>(a.labels) : static_cast<const void *>(a.centres_out);
                dst[i] = pass == 1 ? static_cast<void *>(host_labels[f0 + i]) : static_cast<void *>(host_centres[f0 + i]);
                len[i] = pass == 1 ? sizeof(int32_t) * a.W * a.H : sizeof(float) * 6 * (size_t)a.ns_c * a.ns_r;
                if (!dst[i]) src[i] = nullptr;
            }
        }
        return copy_runs(m, src, dst, len, pass == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, t);
    };
    cudaError_t e = cudaSuccess;
    if (split_groups(b)) {
        // Frame groups: each group's stream copies its frames in, segments
        // them and copies its results out, so one group's copies overlap
        // the other groups' kernels within the call.
        long long n_launch = 0;
        std::string why;
        e = cudaEventRecord(b->ev_fork, s);
        for (int g = 1; g < b->groups && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(b->gstream[g - 1], b->ev_fork, 0);
        for (int g = 0; g < b->groups && e == cudaSuccess; ++g) {
            cudaStream_t t = g == 0 ? s : b->gstream[g - 1];
            const int f0 = b->group_first[g], f1 = b->group_first[g + 1];
            e = copy_frames(f0, f1, 0, t);
            if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("image copy: ") + cudaGetErrorString(e));
            e = enqueue_span(b, span_of(b, g), t, false, n_launch, why);
            if (e != cudaSuccess)
                return bfail(b, SLIC_ERR_CUDA, why.empty() ? std::string("kernel launch: ") + cudaGetErrorString(e) : why);
            for (int pass = 1; pass <= 2 && e == cudaSuccess; ++pass) e = copy_frames(f0, f1, pass, t);
            if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
        }
        for (int g = 1; g < b->groups && e == cudaSuccess; ++g) {
            e = cudaEventRecord(b->ev_join[g - 1], b->gstream[g - 1]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[g - 1], 0);
        }
        if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("stream join: ") + cudaGetErrorString(e));
        b->launches += n_launch;
        return SLIC_OK;
    }
    e = copy_frames(0, n, 0, s);
    if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("image copy: ") + cudaGetErrorString(e));
    const slic_status st = slic_batch_segment(b, stream);
    if (st != SLIC_OK) return st;
    for (int pass = 1; pass <= 2 && e == cudaSuccess; ++pass) e = copy_frames(0, n, pass, s);
    if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

slic_status slic_batch_set_tuning(slic_batch b, int ctas_per_sm, int stages, int rows, int tile_h) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (ctas_per_sm < 0) return bfail(b, SLIC_ERR_INVALID, "ctas_per_sm must be >= 0");
    if (stages != 0 && (stages < 3 || stages > 4)) return bfail(b, SLIC_ERR_INVALID, "stages must be 0, 3 or 4");
    if (rows != 0 && rows != 1 && rows != 2) return bfail(b, SLIC_ERR_INVALID, "rows must be 0, 1 or 2");
    if (tile_h != 0 && tile_h != 32 && tile_h != 64) return bfail(b, SLIC_ERR_INVALID, "tile_h must be 0, 32 or 64");
    if ((rows == 2 || tile_h == 64) && !(b->pipe && b->same8))
        return bfail(b, SLIC_ERR_INVALID, "two row groups and 32x64 tiles need every frame's S to be a multiple of 8");
    const int st = stages ? stages : b->stages, rw = rows ? rows : b->rows, th = tile_h ? tile_h : b->tile_h;
    if (th == 64 && rw != 2) return bfail(b, SLIC_ERR_INVALID, "32x64 tiles need two row groups per warp");
    if ((stages || rows || tile_h) && b->pipe && !shape_fits(b, st, rw, th))
        return bfail(b, SLIC_ERR_INVALID, "the pipeline stages do not fit in shared memory");
    b->ctas_per_sm = ctas_per_sm;
    b->stages = st;
    b->rows = rw;
    b->tile_h = th;
    return SLIC_OK;
}

slic_status slic_batch_set_groups(slic_batch b, int groups) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (groups < 1 || groups > 4 || groups > b->n)
        return bfail(b, SLIC_ERR_INVALID, "groups must be in [1, min(4, n_frames)]");
    if (groups == b->groups) return SLIC_OK;
    for (int g = 0; g + 1 < groups; ++g) {  // internal streams and events, made once
        if (!b->gstream[g] && cudaStreamCreateWithFlags(&b->gstream[g], cudaStreamNonBlocking) != cudaSuccess)
            return bfail(b, SLIC_ERR_CUDA, "cudaStreamCreate failed");
        if (!b->ev_join[g] && cudaEventCreateWithFlags(&b->ev_join[g], cudaEventDisableTiming) != cudaSuccess)
            return bfail(b, SLIC_ERR_CUDA, "cudaEventCreate failed");
    }
    if (groups > 1 && !b->ev_fork && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return bfail(b, SLIC_ERR_CUDA, "cudaEventCreate failed");
    // group g starts at the first frame whose preceding pixels reach g/groups
    // of the batch's pixels (at least one frame per group)
    std::vector<int> first(groups + 1, b->n);
    first[0] = 0;
    long long px = 0;
    int g = 1;
    for (int f = 0; f < b->n && g < groups; ++f) {
        if (f > first[g - 1] && px * groups >= b->total_pixels * g && b->n - f >= groups - g) first[g++] = f;
        px += (long long)b->frames[f].W * b->frames[f].H;
    }
    for (; g < groups; ++g) first[g] = b->n - (groups - g);  // (few frames: the last ones, one each)
    b->group_first = first;
    b->groups = groups;
    if (b->buffers_set) {  // the group tables live in the device tables block
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = upload_tables(b, b->tbl_cur, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
    }
    return SLIC_OK;
}

slic_status slic_batch_set_fused(slic_batch b, int enable) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (enable != 0 && enable != 1) return bfail(b, SLIC_ERR_INVALID, "enable must be 0 or 1");
    b->fused = enable == 1;
    return SLIC_OK;
}

slic_status slic_batch_autotune(slic_batch b, const char *cache_path, void *stream, int *ctas_per_sm, int *stages,
                               int *rows, int *tile_h, int *fused, int *groups) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (!b->buffers_set) return bfail(b, SLIC_ERR_STATE, "slic_batch_set_buffers has not been called");
    const std::string key = tune_key(b);
    int best = 0, best_st = b->stages, best_rw = b->rows, best_th = b->tile_h, best_fu = b->fused ? 1 : 0,
        best_gr = b->groups;
    auto report = [&]() -> slic_status {
        b->ctas_per_sm = best;
        b->stages = best_st;
        b->rows = best_rw;
        b->tile_h = best_th;
        b->fused = best_fu == 1;
        const slic_status r = slic_batch_set_groups(b, best_gr);
        if (r != SLIC_OK) return r;
        if (groups) *groups = best_gr;
        if (ctas_per_sm) *ctas_per_sm = best;
        if (stages) *stages = best_st;
        if (rows) *rows = best_rw;
        if (tile_h) *tile_h = best_th;
        if (fused) *fused = best_fu;
        return SLIC_OK;
    };
    if (cache_path && cache_lookup(cache_path, key, &best, &best_st, &best_rw, &best_th, &best_fu, &best_gr) &&
        best_gr <= b->n && (!b->pipe ? best_rw == 1 && best_th == 32 && best_fu == 0 : shape_fits(b, best_st, best_rw, best_th)))
        return report();
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, SLIC_ERR_CUDA, "cudaEventCreate failed");
    float best_ms = 1e30f;
    slic_status st = SLIC_OK;
    // Search space: frame groups on concurrent streams (1, 2, 4; the plain
    // pipelined path only) x tile shape (32x32, or 32x64 with two row
    // groups) x row groups per warp (pixels per thread and block size) x
    // pipeline stages x resident CTAs per SM (up to what fits) x fused passes
    // or not (one group only).
    const bool can_split = b->pipe && !b->net && b->connectivity != 2;
    const int st_lo = b->pipe ? 3 : b->stages, st_hi = b->pipe ? 4 : b->stages;
    const int rw_hi = (b->pipe && b->same8) ? 2 : 1;
    for (int gr = 1; gr <= (can_split ? std::min(4, b->n) : 1) && st == SLIC_OK; gr *= 2) {
        if ((st = slic_batch_set_groups(b, gr)) != SLIC_OK) break;
        const int fu_hi = b->pipe && b->iterations > 0 && gr == 1 ? 1 : 0;
        for (int th = 32; th <= 64 && st == SLIC_OK; th += 32) {
            for (int rw = 1; rw <= rw_hi && st == SLIC_OK; ++rw) {
                for (int nst = st_lo; nst <= st_hi && st == SLIC_OK; ++nst) {
                    if (b->pipe ? !shape_fits(b, nst, rw, th) : th != 32) continue;
                    const int occ = std::max(b->occupancy, b->pipe ? pipe_occ(b, nst, rw, th) : 0);
                    for (int k = 0; k < occ * (fu_hi + 1) && st == SLIC_OK; ++k) {
                        const int c = 1 + k / (fu_hi + 1), fu = k % (fu_hi + 1);
                        b->ctas_per_sm = c;
                        b->stages = nst;
                        b->rows = rw;
                        b->tile_h = th;
                        b->fused = fu == 1;
                        if ((st = slic_batch_segment(b, stream)) != SLIC_OK) break;  // warm-up
                        float total = 0.0f;
                        for (int rep = 0; rep < 3 && st == SLIC_OK; ++rep) {
                            cudaEventRecord(e0, s);
                            st = slic_batch_segment(b, stream);
                            cudaEventRecord(e1, s);
                            float ms = 0.0f;
                            if (cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                                st = bfail(b, SLIC_ERR_CUDA, "autotune timing failed");
                            total += ms;
                        }
                        if (st == SLIC_OK && total / 3 < best_ms) {
                            best_ms = total / 3;
                            best = c;
                            best_st = nst;
                            best_rw = rw;
                            best_th = th;
                            best_fu = fu;
                            best_gr = gr;
                        }
                    }
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SLIC_OK) return st;
    if ((st = report()) != SLIC_OK) return st;
    if (cache_path) cache_store(cache_path, key, best, best_st, best_rw, best_th, best_fu, best_gr, best_ms);
    return SLIC_OK;
}

slic_status slic_batch_info(slic_batch b, long long *total_pixels, long long *launches, int *ctas_per_sm,
                            int *stages, int *rows, int *tile_h, int *fused, int *groups) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (total_pixels) *total_pixels = b->total_pixels;
    if (launches) *launches = b->launches;
    if (ctas_per_sm)  // resident CTAs per SM of the dominant assignment kernel
        *ctas_per_sm = grid_for(b, b->pipe ? pipe_occ(b, b->stages, b->rows, b->tile_h) : b->occupancy) / b->sms;
    if (stages) *stages = b->pipe ? b->stages : 0;
    if (rows) *rows = b->pipe ? b->rows : 0;
    if (tile_h) *tile_h = b->pipe ? b->tile_h : 32;
    if (fused) *fused = b->pipe && b->fused ? 1 : 0;
    if (groups) *groups = b->groups;
    return SLIC_OK;
}

slic_status slic_batch_profile_enable(slic_batch b, int enable) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (enable && !b->profiling) b->ev_used = 0;
    b->profiling = enable != 0;
    return SLIC_OK;
}

slic_status slic_batch_profile_read(slic_batch b, double *assign_ms, long long *assign_launches) {
    if (!b || !assign_ms || !assign_launches) return bfail(b, SLIC_ERR_INVALID, "NULL argument");
    double total = 0.0;
    for (size_t i = 0; i < b->ev_used; ++i) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(b->events[i].second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->events[i].first, b->events[i].second);
        if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("profile event: ") + cudaGetErrorString(e));
        total += ms;
    }
    *assign_ms = total;
    *assign_launches = (long long)b->ev_used;
    return SLIC_OK;
}

slic_status slic_batch_status(slic_batch b) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    int flag = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (flag) return bfail(b, SLIC_ERR_TIMEOUT, "a bounded wait inside the assignment kernel timed out");
    return SLIC_OK;
}

slic_status slic_batch_iterations_run(slic_batch b, int *out) {
    if (!b || !out) return bfail(b, SLIC_ERR_INVALID, "NULL argument");
    cudaError_t e = cudaDeviceSynchronize();
    for (int f = 0; f < b->n && e == cudaSuccess; ++f) {
        ConvState cs{};
        e = cudaMemcpy(&cs, b->frames[f].cstate, sizeof(ConvState), cudaMemcpyDeviceToHost);
        out[f] = cs.iters;
    }
    if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("state read: ") + cudaGetErrorString(e));
    return SLIC_OK;
}

slic_status slic_batch_profile_times(slic_batch b, double *ms, int max_n, int *n) {
    if (!b || !n || (max_n > 0 && !ms)) return bfail(b, SLIC_ERR_INVALID, "NULL argument");
    const int count = (int)std::min<size_t>(b->ev_used, (size_t)std::max(max_n, 0));
    for (int i = 0; i < count; ++i) {
        float t = 0.0f;
        cudaError_t e = cudaEventSynchronize(b->events[i].second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, b->events[i].first, b->events[i].second);
        if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("profile event: ") + cudaGetErrorString(e));
        ms[i] = t;
    }
    *n = count;
    return SLIC_OK;
}

slic_status slic_batch_grid(slic_batch b, int frame, int *S, int *ns_c, int *ns_r) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (frame < 0 || frame >= b->n) return bfail(b, SLIC_ERR_INVALID, "frame index out of range");
    const FrameArgs &a = b->frames[frame];
    if (S) *S = a.S;
    if (ns_c) *ns_c = a.ns_c;
    if (ns_r) *ns_r = a.ns_r;
    return SLIC_OK;
}

slic_status slic_batch_set_warmstart(slic_batch b, slic_net net) {
    if (!b) return bfail(nullptr, SLIC_ERR_INVALID, "NULL batch");
    if (net) {
        int W = 0, H = 0, S = 0, max_batch = 0;
        float m = 0.0f;
        net_geometry(net, &W, &H, &S, &m, &max_batch);
        for (int f = 0; f < b->n; ++f) {
            const FrameArgs &a = b->frames[f];
            if (a.W != W || a.H != H || a.S != S || b->params[f].m != m)
                return bfail(b, SLIC_ERR_INVALID,
                             "frame " + std::to_string(f) + " differs from the network's width, height, S or m");
            if (a.C != b->frames[0].C) return bfail(b, SLIC_ERR_INVALID, "the frames' channel counts differ");
        }
    }
    // Queued work may still read the tables: wait, then change them.
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && net && !b->net_labels) {
        if (dev_alloc(&b->net_labels, sizeof(int32_t) * (size_t)b->total_pixels) != cudaSuccess) {
            cudaGetLastError();
            b->net_labels = nullptr;
            return bfail(b, SLIC_ERR_NOMEM, "device allocation of the warm-start labels failed");
        }
    }
    if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("device wait: ") + cudaGetErrorString(e));
    b->net = net;
    b->net_C = b->frames[0].C;
    size_t off = 0;
    for (int f = 0; f < b->n; ++f) {
        FrameArgs &a = b->frames[f];
        a.init_labels = net ? b->net_labels + off : nullptr;
        off += (size_t)a.W * a.H;
    }
    if (b->buffers_set) {
        e = upload_tables(b, b->tbl_cur, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return bfail(b, SLIC_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
    }
    return SLIC_OK;
}

const char *slic_batch_last_error(slic_batch b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"
