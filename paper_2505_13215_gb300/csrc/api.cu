// api.cu -- the extern "C" entry points declared in include/splat.h:
// host-side argument checks, per-view parameter packing, workspace carving
// and kernel launches.  No entry point synchronises the stream or reads
// device memory.
#include <atomic>
#include <cmath>

#include "splat_internal.cuh"

namespace splat {

cudaError_t launch_slice_project(const splat_g3&, const splat_g4&, const ViewBatch&, const splat_proj&, int32_t*, int,
                                 const LaunchCtx&);
cudaError_t launch_adjoint(const splat_g3&, const splat_g4&, const ViewBatch&, const splat_proj&, const float*,
                           const splat_grads3&, const splat_grads4&, int32_t*, int, const LaunchCtx&);
cudaError_t launch_bin_sort(const splat_proj&, const ViewBatch&, const splat_bins&, int32_t*, void*, const LaunchCtx&);
size_t bin_sort_workspace(int64_t n_rows, int64_t capacity, int V, const int* TX, const int* TY, int tile_sort);
cudaError_t launch_composite_fwd(const splat_proj&, const splat_bins&, const ViewBatch&, const splat_image&,
                                 const L1Fuse*, int32_t*, int, unsigned long long*, const LaunchCtx&);
cudaError_t launch_composite_bwd(const splat_proj&, const splat_bins&, const ViewBatch&, const splat_image&,
                                 const float*, float*, int32_t*, int, unsigned long long*, const LaunchCtx&);
cudaError_t launch_convert(const splat_g4&, const splat_g3&, float, int64_t*, int32_t*, void*, const LaunchCtx&);
size_t convert_workspace(int64_t n4, int dtype_bytes, int sh_time);
cudaError_t launch_l1_loss(const float*, const float*, int64_t, float, float*, float*, const LaunchCtx&);
cudaError_t launch_convert_state(const splat_g4&, const splat_g3&, float, const splat_adam_set&,
                                 const splat_adam_set&, int32_t*, void*, const LaunchCtx&);
size_t convert_state_workspace(int64_t n4, int sh_time);

constexpr int kMaxSegs = 11;
struct OptSeg {
    float* p;
    float* m;
    float* v;
    const float* g;
    void* st;
    int64_t n;
    float lr;
    float lr_rest;
    int sh;
};
struct OptArgs {
    OptSeg seg[kMaxSegs];
    int nseg;
    int dtype;
    float b1, b2, eps;
    float c1, c2;
    int32_t* status;
};
cudaError_t launch_adam(const OptArgs&, const LaunchCtx&);
cudaError_t launch_cast(const OptArgs&, const LaunchCtx&);

struct StatArgs {
    const float* dproj;
    const uint32_t* n_tiles;
    int64_t N;
    int V;
    float half_w[SPLAT_MAX_VIEWS], half_h[SPLAT_MAX_VIEWS];
    float* accum;
    float* count;
};
struct DensSet {
    int64_t n, capacity;
    float* p[6];
    float* m[6];
    float* v[6];
    const float* accum;
    const float* count;
    const float* noise;
    float* tp[6];
    float* tm[6];
    float* tv[6];
    uint32_t* blocks;
    int64_t* n_out;
    int wsh;
};
struct DensRule {
    float grad_threshold, dense_scale, min_opacity, split_shrink;
};
cudaError_t launch_dens_stats(const StatArgs&, const LaunchCtx&);
cudaError_t launch_densify(const DensSet&, const DensSet&, const DensRule&, void*, int32_t*, const LaunchCtx&);
size_t densify_workspace(int64_t n3, int64_t cap3, int64_t n4, int64_t cap4, int sh_time4);

// Library-wide defaults of the tuning (splat_set_*); a call's splat_options
// overrides them field by field.
static std::atomic<int64_t> g_spin_limit{1ll << 22};
std::atomic<int64_t> g_launches{0};
static std::atomic<int> g_ppl_fwd{8}, g_ppl_bwd{8};
static std::atomic<int> g_tile_sort{0}, g_tile_cull{1};
static std::atomic<unsigned long long*> g_stats{nullptr};
static int g_num_sms[64];

static bool ppl_ok(int p) { return p == 2 || p == 4 || p == 8; }

// A caller's options are valid when every field is its "default" value or in range.
static bool valid_options(const splat_options* o)
{
    if (!o) return true;
    return (o->pixels_per_lane_fwd == 0 || ppl_ok(o->pixels_per_lane_fwd)) &&
           (o->pixels_per_lane_bwd == 0 || ppl_ok(o->pixels_per_lane_bwd)) &&
           o->tile_sort >= -1 && o->tile_sort <= 2 && o->tile_cull >= -1 && o->tile_cull <= 1 &&
           o->spin_limit >= -1;
}

LaunchCtx launch_ctx(void* stream, const splat_options* opt)
{
    LaunchCtx c;
    c.stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (g_num_sms[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        g_num_sms[dev] = n;
    }
    c.num_sms = g_num_sms[dev];
    c.spin_limit = g_spin_limit.load();
    c.tile_sort = g_tile_sort.load();
    c.tile_cull = g_tile_cull.load();
    c.ppl_fwd = g_ppl_fwd.load();
    c.ppl_bwd = g_ppl_bwd.load();
    c.stats = g_stats.load();
    if (opt) {
        if (opt->pixels_per_lane_fwd) c.ppl_fwd = opt->pixels_per_lane_fwd;
        if (opt->pixels_per_lane_bwd) c.ppl_bwd = opt->pixels_per_lane_bwd;
        if (opt->tile_sort >= 0) c.tile_sort = opt->tile_sort;
        if (opt->tile_cull >= 0) c.tile_cull = opt->tile_cull;
        if (opt->spin_limit >= 0) c.spin_limit = opt->spin_limit;
        if (opt->stats) c.stats = opt->stats;
    }
    return c;
}

static bool valid_views(const splat_view* views, int V) { return host_valid_views(views, V); }

static ViewBatch make_batch(const splat_view* views, int V)
{
    ViewBatch b{};
    b.V = V;
    int tiles = 0;
    int64_t pix = 0;
    for (int v = 0; v < V; ++v) {
        const splat_view& s = views[v];
        ViewParams& p = b.v[v];
        for (int k = 0; k < 9; ++k) p.R[k] = s.R[k];
        for (int k = 0; k < 3; ++k) p.T[k] = s.T[k];
        for (int k = 0; k < 3; ++k) p.cam[k] = -(s.R[0 * 3 + k] * s.T[0] + s.R[1 * 3 + k] * s.T[1] + s.R[2 * 3 + k] * s.T[2]);
        p.fx = s.fx; p.fy = s.fy; p.cx = s.cx; p.cy = s.cy;
        p.limx = kFovClamp * (0.5f * (float)s.W / s.fx);
        p.limy = kFovClamp * (0.5f * (float)s.H / s.fy);
        p.t = s.t;
        p.z_near = s.z_near;
        for (int k = 0; k < 3; ++k) p.bg[k] = s.bg[k];
        p.W = s.W; p.H = s.H;
        p.TX = (s.W + kTile - 1) / kTile;
        p.TY = (s.H + kTile - 1) / kTile;
        p.tile_base = tiles;
        p.pix_base = pix;
        tiles += p.TX * p.TY;
        pix += (int64_t)s.W * s.H;
    }
    b.total_tiles = tiles;
    return b;
}

static splat_g3 g3_or_empty(const splat_g3* g)
{
    if (g) return *g;
    splat_g3 e{};
    return e;
}

static splat_g4 g4_or_empty(const splat_g4* g)
{
    if (g) return *g;
    splat_g4 e{};
    return e;
}

static bool valid_g3(const splat_g3& g)
{
    if (g.n < 0) return false;
    if (g.n == 0) return true;
    if (g.dtype < SPLAT_F32 || g.dtype > SPLAT_F16) return false;
    return g.mean && g.log_scale && g.quat && g.opacity && g.sh && g.capacity >= g.n;
}

static bool valid_g4(const splat_g4& g)
{
    if (g.n < 0) return false;
    if (g.n == 0) return true;
    if (g.dtype < SPLAT_F32 || g.dtype > SPLAT_F16) return false;
    if (g.sh_time < 0 || g.sh_time > SPLAT_MAX_SH_TIME) return false;
    return g.mean && g.log_scale && g.ql && g.qr && g.opacity && g.sh;
}

static int common_dtype(const splat_g3& g3, const splat_g4& g4, bool* ok)
{
    *ok = true;
    if (g3.n > 0 && g4.n > 0 && g3.dtype != g4.dtype) *ok = false;
    return g4.n > 0 ? g4.dtype : (g3.n > 0 ? g3.dtype : SPLAT_F32);
}

static bool valid_proj(const splat_proj* p, int V) { return host_valid_proj(p, V); }

static bool aligned(const void* p, size_t a) { return host_aligned(p, a); }

// 16-bit storage: 4-wide rows are read as 8 bytes, SH blocks (96 bytes) as 16-byte vectors
static bool half_storage_aligned(const splat_g3& g3, const splat_g4& g4, int dt)
{
    if (dt == SPLAT_F32) return true;
    if (g4.n > 0 && (!aligned(g4.mean, 8) || !aligned(g4.log_scale, 8) || !aligned(g4.ql, 8) || !aligned(g4.qr, 8) ||
                     !aligned(g4.sh, 16)))
        return false;
    return g3.n == 0 || (aligned(g3.quat, 8) && aligned(g3.sh, 16));
}

static splat_status cuda_status(cudaError_t e) { return e == cudaSuccess ? SPLAT_OK : SPLAT_ERR_CUDA; }

}  // namespace splat

using namespace splat;

extern "C" {

int32_t splat_version(void) { return 0x000100; }

int64_t splat_launch_count(void) { return g_launches.load(); }

void splat_set_spin_limit(int64_t iterations) { g_spin_limit.store(iterations < 0 ? 0 : iterations); }

void splat_set_tile_sort(int mode) { g_tile_sort.store((mode >= 0 && mode <= 2) ? mode : 0); }

void splat_set_stats(unsigned long long* dev_counters) { g_stats.store(dev_counters); }

void splat_set_tile_cull(int on) { g_tile_cull.store(on ? 1 : 0); }

void splat_set_pixels_per_lane(int fwd, int bwd)
{
    if (ppl_ok(fwd)) g_ppl_fwd.store(fwd);
    if (ppl_ok(bwd)) g_ppl_bwd.store(bwd);
}

const char* splat_status_string(int32_t code)
{
    switch (code) {
    case SPLAT_OK: return "ok";
    case SPLAT_ERR_INVALID_ARG: return "invalid argument";
    case SPLAT_ERR_CAPACITY: return "buffer capacity exceeded";
    case SPLAT_ERR_TIMEOUT: return "bounded device wait timed out";
    case SPLAT_ERR_NONFINITE: return "non-finite projected value";
    case SPLAT_ERR_CUDA: return "CUDA error";
    default: return "unknown status";
    }
}

int64_t splat_total_tiles(int V, const int32_t* W, const int32_t* H)
{
    if (!W || !H || V < 0) return -1;
    int64_t t = 0;
    for (int v = 0; v < V; ++v) {
        if (W[v] < 1 || H[v] < 1) return -1;
        t += (int64_t)((W[v] + kTile - 1) / kTile) * ((H[v] + kTile - 1) / kTile);
    }
    return t;
}

size_t splat_workspace_size(int op, int64_t N3, int64_t N4, int V, const int32_t* W, const int32_t* H,
                            int64_t capacity)
{
    return splat_workspace_size_opts(op, N3, N4, V, W, H, capacity, nullptr);
}

size_t splat_workspace_size_opts(int op, int64_t N3, int64_t N4, int V, const int32_t* W, const int32_t* H,
                                 int64_t capacity, const splat_options* opt)
{
    if (N3 < 0 || N4 < 0 || capacity < 0 || capacity > SPLAT_MAX_INSTANCES || !valid_options(opt)) return 0;
    const int tile_sort = (opt && opt->tile_sort >= 0) ? opt->tile_sort : g_tile_sort.load();
    const int64_t N = N3 + N4;
    size_t sort_b = 0, bwd_b = 0, conv_b = 0;
    if (op == SPLAT_OP_BIN_SORT || op == SPLAT_OP_ALL || op == SPLAT_OP_COMPOSITE_BWD) {
        if (V < 1 || V > SPLAT_MAX_VIEWS || splat_total_tiles(V, W, H) < 0) return 0;
    }
    if (op == SPLAT_OP_BIN_SORT || op == SPLAT_OP_ALL) {
        int TX[SPLAT_MAX_VIEWS], TY[SPLAT_MAX_VIEWS];
        for (int v = 0; v < V; ++v) {
            TX[v] = (W[v] + kTile - 1) / kTile;
            TY[v] = (H[v] + kTile - 1) / kTile;
        }
        sort_b = bin_sort_workspace(N * V, capacity, V, TX, TY, tile_sort);
    }
    if (op == SPLAT_OP_COMPOSITE_BWD || op == SPLAT_OP_ALL) bwd_b = ((size_t)N * V * 48 + 255) & ~(size_t)255;
    if (op == SPLAT_OP_CONVERT || op == SPLAT_OP_ALL) conv_b = convert_workspace(N4, 4, 0);
    size_t state_b = 0;
    if (op == SPLAT_OP_CONVERT_STATE || op == SPLAT_OP_ALL) state_b = convert_state_workspace(N4, 0);
    if (op < SPLAT_OP_BIN_SORT || op > SPLAT_OP_CONVERT_STATE) return 0;
    size_t m = sort_b;
    if (bwd_b > m) m = bwd_b;
    if (conv_b > m) m = conv_b;
    if (state_b > m) m = state_b;
    return m < 256 ? 256 : m;
}

splat_status splat_slice_project(const splat_g3* g3p, const splat_g4* g4p, const splat_view* views, int V,
                                 splat_proj* out, int32_t* status, void* stream)
{
    const splat_g3 g3 = g3_or_empty(g3p);
    const splat_g4 g4 = g4_or_empty(g4p);
    bool same = true;
    const int dt = common_dtype(g3, g4, &same);
    if (!same || !valid_g3(g3) || !valid_g4(g4) || !valid_views(views, V) || !valid_proj(out, V) || !status)
        return SPLAT_ERR_INVALID_ARG;
    if (out->n != g3.n + g4.n) return SPLAT_ERR_INVALID_ARG;
    if (!aligned(out->conic_opacity, 16) || !aligned(out->rgb_depth, 16) || !aligned(out->rect, 16) ||
        !aligned(out->xy, 8))
        return SPLAT_ERR_INVALID_ARG;
    if (g4.n > 0 && dt == SPLAT_F32 && (!aligned(g4.mean, 16) || !aligned(g4.log_scale, 16) || !aligned(g4.ql, 16) ||
                                        !aligned(g4.qr, 16) || !aligned(g4.sh, 16)))
        return SPLAT_ERR_INVALID_ARG;
    if (g3.n > 0 && dt == SPLAT_F32 && (!aligned(g3.quat, 16) || !aligned(g3.sh, 16))) return SPLAT_ERR_INVALID_ARG;
    if (!half_storage_aligned(g3, g4, dt)) return SPLAT_ERR_INVALID_ARG;
    const LaunchCtx ctx = launch_ctx(stream);
    cudaError_t e = cudaMemsetAsync(status, 0, 4 * sizeof(int32_t), ctx.stream);
    if (e != cudaSuccess) return SPLAT_ERR_CUDA;
    const ViewBatch vb = make_batch(views, V);
    return cuda_status(launch_slice_project(g3, g4, vb, *out, status, dt, ctx));
}

splat_status splat_bin_sort(const splat_proj* proj, const splat_view* views, int V, splat_bins* bins,
                            int32_t* status, void* workspace, size_t workspace_bytes, void* stream)
{
    return splat_bin_sort_opts(proj, views, V, bins, status, workspace, workspace_bytes, nullptr, stream);
}

splat_status splat_bin_sort_opts(const splat_proj* proj, const splat_view* views, int V, splat_bins* bins,
                                 int32_t* status, void* workspace, size_t workspace_bytes, const splat_options* opt,
                                 void* stream)
{
    if (!valid_views(views, V) || !valid_proj(proj, V) || !host_valid_bins(bins) || !status || !valid_options(opt))
        return SPLAT_ERR_INVALID_ARG;
    int TX[SPLAT_MAX_VIEWS], TY[SPLAT_MAX_VIEWS];
    for (int v = 0; v < V; ++v) {
        TX[v] = (views[v].W + kTile - 1) / kTile;
        TY[v] = (views[v].H + kTile - 1) / kTile;
    }
    const LaunchCtx ctx = launch_ctx(stream, opt);
    const size_t need = bin_sort_workspace(proj->n * V, bins->capacity, V, TX, TY, ctx.tile_sort);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return SPLAT_ERR_INVALID_ARG;
    const ViewBatch vb = make_batch(views, V);
    return cuda_status(launch_bin_sort(*proj, vb, *bins, status, workspace, ctx));
}

splat_status splat_composite_fwd(const splat_proj* proj, const splat_bins* bins, const splat_view* views, int V,
                                 splat_image* img, int32_t* status, void* stream)
{
    return splat_composite_fwd_opts(proj, bins, views, V, img, status, nullptr, stream);
}

splat_status splat_composite_fwd_opts(const splat_proj* proj, const splat_bins* bins, const splat_view* views, int V,
                                      splat_image* img, int32_t* status, const splat_options* opt, void* stream)
{
    if (!valid_views(views, V) || !valid_proj(proj, V) || !bins || !img || !status || !valid_options(opt))
        return SPLAT_ERR_INVALID_ARG;
    if (!img->rgb || !img->final_T || !img->last || !bins->ranges || (bins->capacity > 0 && !bins->vals))
        return SPLAT_ERR_INVALID_ARG;
    const LaunchCtx ctx = launch_ctx(stream, opt);
    const ViewBatch vb = make_batch(views, V);
    return cuda_status(launch_composite_fwd(*proj, *bins, vb, *img, nullptr, status, ctx.ppl_fwd, ctx.stats, ctx));
}

splat_status splat_composite_fwd_l1(const splat_proj* proj, const splat_bins* bins, const splat_view* views, int V,
                                    splat_image* img, const float* target, float scale, float* dL_drgb, float* loss,
                                    int32_t* status, void* stream)
{
    return splat_composite_fwd_l1_opts(proj, bins, views, V, img, target, scale, dL_drgb, loss, status, nullptr,
                                       stream);
}

splat_status splat_composite_fwd_l1_opts(const splat_proj* proj, const splat_bins* bins, const splat_view* views,
                                         int V, splat_image* img, const float* target, float scale, float* dL_drgb,
                                         float* loss, int32_t* status, const splat_options* opt, void* stream)
{
    if (!valid_views(views, V) || !valid_proj(proj, V) || !bins || !img || !status || !valid_options(opt))
        return SPLAT_ERR_INVALID_ARG;
    if (!img->rgb || !img->final_T || !img->last || !bins->ranges || (bins->capacity > 0 && !bins->vals))
        return SPLAT_ERR_INVALID_ARG;
    if (!target || !dL_drgb || !loss || !std::isfinite(scale)) return SPLAT_ERR_INVALID_ARG;
    const LaunchCtx ctx = launch_ctx(stream, opt);
    const ViewBatch vb = make_batch(views, V);
    const L1Fuse l1{target, scale, dL_drgb, loss};
    return cuda_status(launch_composite_fwd(*proj, *bins, vb, *img, &l1, status, ctx.ppl_fwd, ctx.stats, ctx));
}

splat_status splat_composite_bwd(const splat_proj* proj, const splat_bins* bins, const splat_view* views, int V,
                                 const splat_image* img, const float* dL_drgb, const splat_g3* g3p, const splat_g4* g4p,
                                 splat_grads3* dg3, splat_grads4* dg4, float* dproj, uint32_t flags, int32_t* status,
                                 void* workspace, size_t workspace_bytes, void* stream)
{
    return splat_composite_bwd_opts(proj, bins, views, V, img, dL_drgb, g3p, g4p, dg3, dg4, dproj, flags, status,
                                    workspace, workspace_bytes, nullptr, stream);
}

splat_status splat_composite_bwd_opts(const splat_proj* proj, const splat_bins* bins, const splat_view* views, int V,
                                      const splat_image* img, const float* dL_drgb, const splat_g3* g3p,
                                      const splat_g4* g4p, splat_grads3* dg3, splat_grads4* dg4, float* dproj,
                                      uint32_t flags, int32_t* status, void* workspace, size_t workspace_bytes,
                                      const splat_options* opt, void* stream)
{
    if (!valid_options(opt)) return SPLAT_ERR_INVALID_ARG;
    const splat_g3 g3 = g3_or_empty(g3p);
    const splat_g4 g4 = g4_or_empty(g4p);
    bool same = true;
    const int dt = common_dtype(g3, g4, &same);
    const bool stop2d = (flags & SPLAT_BWD_STOP_2D) != 0;
    const bool adj_only = (flags & SPLAT_BWD_ADJOINT_ONLY) != 0;
    if (!same || !valid_views(views, V) || !valid_proj(proj, V) || !status || (stop2d && adj_only))
        return SPLAT_ERR_INVALID_ARG;
    if (!adj_only && (!bins || !img || !dL_drgb || !img->final_T || !img->last || !bins->ranges))
        return SPLAT_ERR_INVALID_ARG;
    if (adj_only && !dproj) return SPLAT_ERR_INVALID_ARG;
    if (dproj && !aligned(dproj, 16)) return SPLAT_ERR_INVALID_ARG;
    if (!stop2d) {
        if (!valid_g3(g3) || !valid_g4(g4) || proj->n != g3.n + g4.n) return SPLAT_ERR_INVALID_ARG;
        if (g3.n > 0 && (!dg3 || !dg3->mean || !dg3->log_scale || !dg3->quat || !dg3->opacity || !dg3->sh))
            return SPLAT_ERR_INVALID_ARG;
        if (g4.n > 0 && (!dg4 || !dg4->mean || !dg4->log_scale || !dg4->ql || !dg4->qr || !dg4->opacity || !dg4->sh))
            return SPLAT_ERR_INVALID_ARG;
        if (g4.n > 0 && (!aligned(dg4->mean, 16) || !aligned(dg4->log_scale, 16) || !aligned(dg4->ql, 16) ||
                         !aligned(dg4->qr, 16) || !aligned(dg4->sh, 16)))
            return SPLAT_ERR_INVALID_ARG;
        if (g3.n > 0 && (!aligned(dg3->quat, 16) || !aligned(dg3->sh, 16))) return SPLAT_ERR_INVALID_ARG;
        if (g4.n > 0 && dt == SPLAT_F32 && (!aligned(g4.mean, 16) || !aligned(g4.ql, 16) || !aligned(g4.qr, 16) ||
                                            !aligned(g4.log_scale, 16) || !aligned(g4.sh, 16)))
            return SPLAT_ERR_INVALID_ARG;
        if (g3.n > 0 && dt == SPLAT_F32 && (!aligned(g3.quat, 16) || !aligned(g3.sh, 16))) return SPLAT_ERR_INVALID_ARG;
        if (!half_storage_aligned(g3, g4, dt)) return SPLAT_ERR_INVALID_ARG;
    }
    const size_t dproj_bytes = (size_t)proj->n * V * 48;
    float* dp = dproj;
    if (!dp) {
        if (!workspace || workspace_bytes < dproj_bytes || !aligned(workspace, 256)) return SPLAT_ERR_INVALID_ARG;
        dp = (float*)workspace;
    } else if (!aligned(dp, 16)) {
        return SPLAT_ERR_INVALID_ARG;
    }
    const LaunchCtx ctx = launch_ctx(stream, opt);
    const ViewBatch vb = make_batch(views, V);
    if (!adj_only) {
        cudaError_t e = cudaMemsetAsync(dp, 0, dproj_bytes, ctx.stream);
        if (e != cudaSuccess) return SPLAT_ERR_CUDA;
        e = launch_composite_bwd(*proj, *bins, vb, *img, dL_drgb, dp, status, ctx.ppl_bwd, ctx.stats, ctx);
        if (e != cudaSuccess) return SPLAT_ERR_CUDA;
    }
    if (stop2d) return SPLAT_OK;
    splat_grads3 d3 = dg3 ? *dg3 : splat_grads3{};
    splat_grads4 d4 = dg4 ? *dg4 : splat_grads4{};
    return cuda_status(launch_adjoint(g3, g4, vb, *proj, dp, d3, d4, status, dt, ctx));
}

splat_status splat_convert_4d_to_3d(splat_g4* g4, splat_g3* g3, float tau, int64_t* n_moved_dev, int32_t* status,
                                    void* workspace, size_t workspace_bytes, void* stream)
{
    if (!g4 || !g3 || !n_moved_dev || !status || !std::isfinite(tau)) return SPLAT_ERR_INVALID_ARG;
    if (!valid_g4(*g4) || g3->n < 0 || g3->capacity < g3->n) return SPLAT_ERR_INVALID_ARG;
    if (g4->n > 0 && (!g3->mean || !g3->log_scale || !g3->quat || !g3->opacity || !g3->sh)) return SPLAT_ERR_INVALID_ARG;
    if (g4->n > 0 && g3->dtype != g4->dtype) return SPLAT_ERR_INVALID_ARG;
    if (g4->n > 0 && g4->dtype == SPLAT_F32 && (!aligned(g4->ql, 16) || !aligned(g4->qr, 16)))
        return SPLAT_ERR_INVALID_ARG;
    const int bytes = g4->dtype == SPLAT_F32 ? 4 : 2;
    const size_t need = convert_workspace(g4->n, bytes, g4->sh_time);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return SPLAT_ERR_INVALID_ARG;
    const LaunchCtx ctx = launch_ctx(stream);
    return cuda_status(launch_convert(*g4, *g3, tau, n_moved_dev, status, workspace, ctx));
}

static const int kWidth3[5] = {3, 3, 4, 1, 48};
// floats per row of a 4D field; sh holds a block of 48 per time frequency
static int width4(int f, int sh_time) { return f < 4 ? 4 : (f == 4 ? 1 : 48 * (sh_time + 1)); }

static bool valid_set(const splat_adam_set* s, int fields, int64_t rows, bool need_param, bool need_moments)
{
    if (rows == 0) return true;
    if (!s) return false;
    for (int f = 0; f < fields; ++f) {
        if (need_param && (!s->param[f] || !aligned(s->param[f], 16))) return false;
        if (need_moments && (!s->m[f] || !s->v[f] || !aligned(s->m[f], 16) || !aligned(s->v[f], 16))) return false;
    }
    return true;
}

static void* field3(const splat_g3& g, int f)
{
    void* p[5] = {g.mean, g.log_scale, g.quat, g.opacity, g.sh};
    return p[f];
}

static void* field4(const splat_g4& g, int f)
{
    void* p[6] = {g.mean, g.log_scale, g.ql, g.qr, g.opacity, g.sh};
    return p[f];
}

splat_status splat_adam_step(const splat_adam_hyper* h, splat_adam_set* s3, const splat_grads3* dg3, splat_g3* g3,
                             splat_adam_set* s4, const splat_grads4* dg4, splat_g4* g4, int32_t* status, void* stream)
{
    if (!h || !g3 || !g4 || !status || h->step < 1) return SPLAT_ERR_INVALID_ARG;
    if (g4->sh_time < 0 || g4->sh_time > SPLAT_MAX_SH_TIME) return SPLAT_ERR_INVALID_ARG;
    if (g3->n < 0 || g4->n < 0 || g3->capacity < g3->n || g3->dtype != g4->dtype) return SPLAT_ERR_INVALID_ARG;
    if (g3->dtype < SPLAT_F32 || g3->dtype > SPLAT_F16) return SPLAT_ERR_INVALID_ARG;
    if (!(h->beta1 >= 0.f && h->beta1 < 1.f) || !(h->beta2 >= 0.f && h->beta2 < 1.f) || !(h->eps > 0.f))
        return SPLAT_ERR_INVALID_ARG;
    if (!valid_set(s3, 5, g3->n, true, true) || !valid_set(s4, 6, g4->n, true, true)) return SPLAT_ERR_INVALID_ARG;
    if ((g3->n > 0 && !dg3) || (g4->n > 0 && !dg4)) return SPLAT_ERR_INVALID_ARG;
    OptArgs a{};
    const float* gr3[5] = {};
    const float* gr4[6] = {};
    if (dg3) {
        gr3[0] = dg3->mean; gr3[1] = dg3->log_scale; gr3[2] = dg3->quat; gr3[3] = dg3->opacity; gr3[4] = dg3->sh;
    }
    if (dg4) {
        gr4[0] = dg4->mean; gr4[1] = dg4->log_scale; gr4[2] = dg4->ql; gr4[3] = dg4->qr; gr4[4] = dg4->opacity;
        gr4[5] = dg4->sh;
    }
    for (int f = 0; f < 5 && g3->n > 0; ++f) {
        if (!gr3[f] || !field3(*g3, f) || !std::isfinite(h->lr3[f])) return SPLAT_ERR_INVALID_ARG;
        a.seg[a.nseg++] = OptSeg{s3->param[f], s3->m[f], s3->v[f], gr3[f], field3(*g3, f), g3->n * kWidth3[f],
                                 h->lr3[f], h->lr_sh_rest, f == 4 ? 48 : 0};
    }
    for (int f = 0; f < 6 && g4->n > 0; ++f) {
        if (!gr4[f] || !field4(*g4, f) || !std::isfinite(h->lr4[f])) return SPLAT_ERR_INVALID_ARG;
        a.seg[a.nseg++] = OptSeg{s4->param[f], s4->m[f], s4->v[f], gr4[f], field4(*g4, f),
                                 g4->n * width4(f, g4->sh_time), h->lr4[f], h->lr_sh_rest,
                                 f == 5 ? width4(5, g4->sh_time) : 0};
    }
    if (!std::isfinite(h->lr_sh_rest)) return SPLAT_ERR_INVALID_ARG;
    a.dtype = g3->dtype;
    a.b1 = h->beta1;
    a.b2 = h->beta2;
    a.eps = h->eps;
    a.c1 = (float)(1.0 / (1.0 - std::pow((double)h->beta1, (double)h->step)));
    a.c2 = (float)(1.0 / (1.0 - std::pow((double)h->beta2, (double)h->step)));
    a.status = status;
    const LaunchCtx ctx = launch_ctx(stream);
    return cuda_status(launch_adam(a, ctx));
}

splat_status splat_cast_params(const splat_g3* src3, splat_g3* dst3, const splat_g4* src4, splat_g4* dst4,
                               void* stream)
{
    if (!src3 || !dst3 || !src4 || !dst4) return SPLAT_ERR_INVALID_ARG;
    if (src3->dtype != SPLAT_F32 || src4->dtype != SPLAT_F32 || dst3->dtype != dst4->dtype) return SPLAT_ERR_INVALID_ARG;
    if (dst3->dtype < SPLAT_F32 || dst3->dtype > SPLAT_F16 || src3->n < 0 || src4->n < 0) return SPLAT_ERR_INVALID_ARG;
    if (src4->sh_time != dst4->sh_time || src4->sh_time < 0 || src4->sh_time > SPLAT_MAX_SH_TIME)
        return SPLAT_ERR_INVALID_ARG;
    if (src3->n > dst3->capacity) return SPLAT_ERR_INVALID_ARG;
    OptArgs a{};
    for (int f = 0; f < 5 && src3->n > 0; ++f) {
        if (!field3(*src3, f) || !field3(*dst3, f)) return SPLAT_ERR_INVALID_ARG;
        a.seg[a.nseg++] = OptSeg{(float*)field3(*src3, f), nullptr, nullptr, nullptr, field3(*dst3, f),
                                 src3->n * kWidth3[f], 0.f, 0.f, 0};
    }
    for (int f = 0; f < 6 && src4->n > 0; ++f) {
        if (!field4(*src4, f) || !field4(*dst4, f)) return SPLAT_ERR_INVALID_ARG;
        a.seg[a.nseg++] = OptSeg{(float*)field4(*src4, f), nullptr, nullptr, nullptr, field4(*dst4, f),
                                 src4->n * width4(f, src4->sh_time), 0.f, 0.f, 0};
    }
    a.dtype = dst3->dtype;
    const LaunchCtx ctx = launch_ctx(stream);
    return cuda_status(launch_cast(a, ctx));
}

splat_status splat_convert_adam_state(const splat_g4* g4, const splat_g3* g3, float tau, splat_adam_set* s4,
                                      splat_adam_set* s3, int32_t* status, void* workspace, size_t workspace_bytes,
                                      void* stream)
{
    if (!g4 || !g3 || !status || !std::isfinite(tau)) return SPLAT_ERR_INVALID_ARG;
    if (!valid_g4(*g4) || g3->n < 0 || g3->capacity < g3->n) return SPLAT_ERR_INVALID_ARG;
    if (!valid_set(s4, 6, g4->n, false, true)) return SPLAT_ERR_INVALID_ARG;
    if (g4->n > 0 && !valid_set(s3, 5, g3->capacity, false, true)) return SPLAT_ERR_INVALID_ARG;
    const size_t need = convert_state_workspace(g4->n, g4->sh_time);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return SPLAT_ERR_INVALID_ARG;
    const LaunchCtx ctx = launch_ctx(stream);
    const splat_adam_set empty{};
    return cuda_status(launch_convert_state(*g4, *g3, tau, s4 ? *s4 : empty, s3 ? *s3 : empty, status, workspace, ctx));
}

splat_status splat_densify_stats(const splat_proj* proj, const splat_view* views, int V, const float* dproj,
                                 float* accum, float* count, void* stream)
{
    if (!valid_views(views, V) || !valid_proj(proj, V) || proj->n < 0) return SPLAT_ERR_INVALID_ARG;
    if (proj->n > 0 && (!proj->n_tiles || !dproj || !accum || !count || !aligned(dproj, 16)))
        return SPLAT_ERR_INVALID_ARG;
    StatArgs a{};
    a.dproj = dproj;
    a.n_tiles = (const uint32_t*)proj->n_tiles;
    a.N = proj->n;
    a.V = V;
    for (int v = 0; v < V; ++v) {
        a.half_w[v] = 0.5f * (float)views[v].W;
        a.half_h[v] = 0.5f * (float)views[v].H;
    }
    a.accum = accum;
    a.count = count;
    const LaunchCtx ctx = launch_ctx(stream);
    return cuda_status(launch_dens_stats(a, ctx));
}

size_t splat_densify_workspace_size(int64_t n3, int64_t capacity3, int64_t n4, int64_t capacity4, int sh_time4)
{
    if (n3 < 0 || n4 < 0 || capacity3 < n3 || capacity4 < n4 || sh_time4 < 0 || sh_time4 > SPLAT_MAX_SH_TIME) return 0;
    return densify_workspace(n3, capacity3, n4, capacity4, sh_time4);
}

size_t splat_workspace_size_4d(int op, int64_t N4, int sh_time)
{
    if (N4 < 0 || sh_time < 0 || sh_time > SPLAT_MAX_SH_TIME) return 0;
    if (op == SPLAT_OP_CONVERT) return convert_workspace(N4, 4, sh_time);
    if (op == SPLAT_OP_CONVERT_STATE) return convert_state_workspace(N4, sh_time);
    return 0;
}

static bool dens_set_ok(const splat_densify_set* s, int fields)
{
    if (!s || s->n < 0 || s->capacity < s->n || s->sh_time < 0 || s->sh_time > SPLAT_MAX_SH_TIME) return false;
    if (fields == 5 && s->sh_time != 0) return false;
    if (s->n == 0) return true;
    if (!s->accum || !s->count || !s->noise || !valid_set(s->state, fields, s->n, true, true)) return false;
    return true;
}

static DensSet dens_set_of(const splat_densify_set& s, int fields, int64_t* n_out)
{
    DensSet d{};
    d.n = s.n;
    d.capacity = s.capacity;
    for (int f = 0; f < fields && s.n > 0; ++f) {
        d.p[f] = s.state->param[f];
        d.m[f] = s.state->m[f];
        d.v[f] = s.state->v[f];
    }
    d.accum = s.accum;
    d.count = s.count;
    d.noise = s.noise;
    d.n_out = n_out;
    d.wsh = 48 * (s.sh_time + 1);
    return d;
}

splat_status splat_densify(const splat_densify_rule* rule, splat_densify_set* set3, splat_densify_set* set4,
                           int64_t* n_out, int32_t* status, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!rule || !n_out || !status || !dens_set_ok(set3, 5) || !dens_set_ok(set4, 6)) return SPLAT_ERR_INVALID_ARG;
    if (!std::isfinite(rule->grad_threshold) || !std::isfinite(rule->dense_scale) ||
        !std::isfinite(rule->min_opacity) || !std::isfinite(rule->split_shrink))
        return SPLAT_ERR_INVALID_ARG;
    const size_t need = densify_workspace(set3->n, set3->capacity, set4->n, set4->capacity, set4->sh_time);
    if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return SPLAT_ERR_INVALID_ARG;
    const DensRule r{rule->grad_threshold, rule->dense_scale, rule->min_opacity, rule->split_shrink};
    const LaunchCtx ctx = launch_ctx(stream);
    return cuda_status(launch_densify(dens_set_of(*set3, 5, n_out), dens_set_of(*set4, 6, n_out + 1), r, workspace,
                                      status, ctx));
}

splat_status splat_l1_loss(const float* img, const float* target, int64_t n, float scale, float* dL_dimg,
                           float* loss, void* stream)
{
    if (n < 0 || !loss || (n > 0 && (!img || !target || !dL_dimg)) || !std::isfinite(scale)) return SPLAT_ERR_INVALID_ARG;
    if (!aligned(img, 16) || !aligned(target, 16) || !aligned(dL_dimg, 16)) return SPLAT_ERR_INVALID_ARG;
    const LaunchCtx ctx = launch_ctx(stream);
    return cuda_status(launch_l1_loss(img, target, n, scale, dL_dimg, loss, ctx));
}

}  // extern "C"
