// alf_api.cu -- the C ABI declared in include/alifmm.h: validation, plan
// layout (fields, tiles, work queue), workspace ownership and launch order.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "alf_internal.h"

// CTAs per SM of the FP64 check: enough warps for the FP64 pipe, room left for other streams'
// kernels (rays, adjoint) on the same SMs
#define ALF_CHECK_CTAS_PER_SM 2

using namespace alf;

namespace {

alf_status fail(alf_ctx* ctx, alf_status code, const char* fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

#define ALF_CUDA(ctx, call)                                                                              \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            if (e_ == cudaErrorMemoryAllocation)                                                         \
                return fail(ctx, ALF_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_));                  \
            return fail(ctx, ALF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                     \
        }                                                                                                \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n)
{
    return cudaMalloc((void**)p, std::max<size_t>(1, n) * sizeof(T));
}

void dfree(void* p)
{
    if (p) cudaFree(p);
}

// The constants of one material for wave mode `mode` (0 qP, 1 qSV, 2 SH; see MatD).  False for a
// non-physical material.
bool material_to_matd(const alf_material& m, int mode, MatD* out)
{
    const double c22 = m.c[1][1], c23 = m.c[1][2], c33 = m.c[2][2], c44 = m.c[3][3], rho = m.rho;
    const double c55 = m.c[4][4], c66 = m.c[5][5];
    if (!(rho > 0.0) || !std::isfinite(rho)) return false;
    for (double v : {c22, c23, c33, c44})
        if (!std::isfinite(v)) return false;
    // the in-plane stiffness (c22, c23; c23, c33 and the shear c44) must be positive definite: the
    // Christoffel matrix is then positive definite in every direction, so both of its eigenvalues
    // (qP and qSV lambda, Sec. 3.2) are > 0
    if (!(c22 > 0.0 && c33 > 0.0 && c44 > 0.0)) return false;
    if (!(c22 * c33 - c23 * c23 > 0.0)) return false;
    *out = MatD{};
    out->a22 = c22 / rho;
    out->a23 = c23 / rho;
    out->a33 = c33 / rho;
    out->a44 = c44 / rho;
    out->iso = (c22 == c33 && c23 == c22 - 2.0 * c44) ? 1 : 0;
    if (mode == 1) {
        out->sv = 1;
        if (out->iso) out->a22 = c44 / rho;  // an isotropic solid's shear speed
    } else if (mode == 2) {
        // SH: the out-of-plane eigenvalue c66 cos^2 + c55 sin^2
        if (!(c55 > 0.0 && c66 > 0.0) || !std::isfinite(c55) || !std::isfinite(c66)) return false;
        out->a22 = c66 / rho;
        out->a33 = c55 / rho;
        out->a44 = 0.0;
        out->a23 = std::sqrt(out->a22 * out->a33);
        out->iso = c55 == c66 ? 1 : 0;
    }
    return true;
}

// lambda / rho of a material's mode at phase angle th (host copy of the device formula)
double mode_lambda_host(const MatD& m, double th)
{
    if (m.iso) return m.a22;
    const double c = std::cos(th), sn = std::sin(th);
    const double al = c * c * m.a22 + sn * sn * m.a44, ga = c * c * m.a44 + sn * sn * m.a33;
    const double be = c * sn * (m.a23 + m.a44);
    const double r = std::sqrt((al - ga) * (al - ga) + 4.0 * be * be);
    return 0.5 * ((al + ga) + (m.sv ? -r : r));
}


cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }


// The sweep rounds until every dirty set is empty.  Rounds are issued in
// chunks of rounds_per_check (an even number, so every chunk starts at parity
// 0); after each chunk the remaining work is read back.  A chunk is replayed
// from a CUDA graph captured for the current output pointers, unless the
// evaluation kernel is being timed.
alf_status run_sweep(alf_plan* p, const FimLaunch& a, cudaStream_t st)
{
    alf_ctx* ctx = p->ctx;
    const int prec = p->opt.precision;
    long long max_total = 0;
    for (const FieldDesc& fd : p->fields) max_total = std::max(max_total, (long long)(fd.nx + fd.ny));
    max_total *= p->opt.max_rounds;
    const bool timing = p->opt.time_kernels != 0;
    // stream capture is not possible on the legacy default stream: launch directly there
    const bool graph = p->opt.use_graph != 0 && !timing && st != nullptr && st != cudaStreamLegacy &&
                       st != cudaStreamPerThread;
    if (timing && p->ev.empty()) {
        p->ev.resize(2 * (size_t)p->rounds_per_check);
        for (auto& e : p->ev) ALF_CUDA(ctx, cudaEventCreate(&e));
    }
    p->eval_ms = 0.0;
    p->eval_launches = 0;
    p->sweep_rounds = 0;
    if (graph && (p->chunk_graph == nullptr || p->graph_times != a.times || p->graph_records != a.records)) {
        if (p->chunk_graph) {
            cudaGraphExecDestroy(p->chunk_graph);
            p->chunk_graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        ALF_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = cudaSuccess;
        for (int k = 0; k < p->rounds_per_check && ce == cudaSuccess; ++k)
            ce = launch_fim_round(prec, a, k & 1, p->grid_fields, p->grid_eval, st, p->eval_block);
        if (ce == cudaSuccess) ce = launch_fim_pending(a, 0, p->d_pending, st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(p->h_pending, p->d_pending, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        cudaError_t ee = cudaStreamEndCapture(st, &g);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(ctx, ALF_ERR_CUDA, "sweep graph capture: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        }
        ee = cudaGraphInstantiate(&p->chunk_graph, g, 0);
        cudaGraphDestroy(g);
        if (ee != cudaSuccess) return fail(ctx, ALF_ERR_CUDA, "sweep graph: %s", cudaGetErrorString(ee));
        p->graph_times = a.times;
        p->graph_records = a.records;
    }
    for (long long r = 0; r < max_total;) {
        if (graph) {
            ALF_CUDA(ctx, cudaGraphLaunch(p->chunk_graph, st));
            note_launches((unsigned)p->rounds_per_check * 4 + 1);
            r += p->rounds_per_check;
        } else {
            for (int k = 0; k < p->rounds_per_check; ++k, ++r) {
                cudaEvent_t e0 = timing ? p->ev[2 * k] : nullptr, e1 = timing ? p->ev[2 * k + 1] : nullptr;
                ALF_CUDA(ctx, launch_fim_round(prec, a, k & 1, p->grid_fields, p->grid_eval, st, p->eval_block, e0, e1));
            }
            ALF_CUDA(ctx, launch_fim_pending(a, 0, p->d_pending, st));
            ALF_CUDA(ctx, cudaMemcpyAsync(p->h_pending, p->d_pending, sizeof(unsigned long long),
                                          cudaMemcpyDeviceToHost, st));
        }
        ALF_CUDA(ctx, cudaStreamSynchronize(st));
        p->sweep_rounds += (unsigned long long)p->rounds_per_check;
        if (timing)
            for (int k = 0; k < p->rounds_per_check; ++k) {
                float ms = 0.f;
                ALF_CUDA(ctx, cudaEventElapsedTime(&ms, p->ev[2 * k], p->ev[2 * k + 1]));
                p->eval_ms += ms;
                p->eval_launches++;
            }
        if (*p->h_pending == 0ull) break;
    }
    // the cap ended the loop with work left: some field never reached its fixed point
    if (*p->h_pending != 0ull) ALF_CUDA(ctx, launch_set_status(p->d_q, ALF_ERR_NOT_CONVERGED, st));
    return ALF_OK;
}

}  // namespace

// CTA-per-field sweep shape: threads per CTA, CTAs per field (a cluster) and a grid of as many CTAs as are
// resident at once; a cluster that cannot be resident falls back to one CTA per field
static void set_cta_shape(alf_plan* p, int threads, int cluster, int precision, bool vtable)
{
    if (cluster > 1 && fim_cta_grid(precision, p->cta_words, vtable, 512, cluster, p->ctx->nsm) < cluster) cluster = 1;
    p->cta_threads = cluster > 1 ? 512 : threads;
    p->cta_cluster = cluster;
    p->cta_grid = std::max(p->cta_cluster,
                           fim_cta_grid(precision, p->cta_words, vtable, p->cta_threads, cluster, p->ctx->nsm));
}

extern "C" {

void alf_default_options(alf_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = ALF_FP32;
    o->group_model = ALF_GROUP_PAPER;
    o->init_mode = ALF_INIT_RADIUS;
    o->init_radius = 2;
    o->n_levels = 3;
    o->level_density[0] = 27;
    o->level_density[1] = 9;
    o->level_density[2] = 3;
    o->level_radius[0] = 1;
    o->level_radius[1] = 6;
    o->level_radius[2] = 13;
    o->plane_step = 4;
    o->ray_halfwidth = 8;
    o->stop_radius = 1.6;
    o->max_ray_points = 512;
    o->max_rounds = 64;
    o->sweep = 0;
    o->ray_family = 0;
    o->keep_records = 0;
    o->band_cells = 2.0;
    o->use_graph = 1;
    o->time_kernels = 0;
    o->subgrid = 1;
    o->wave_mode = 0;
}

alf_status alf_create(alf_ctx** out, int cuda_device)
{
    if (!out) return ALF_ERR_INVALID_ARG;
    *out = nullptr;
    alf_ctx* ctx = new (std::nothrow) alf_ctx();
    if (!ctx) return ALF_ERR_OOM;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || cuda_device < 0 || cuda_device >= n) {
        delete ctx;
        return ALF_ERR_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaSetDevice(cuda_device) != cudaSuccess || cudaGetDeviceProperties(&prop, cuda_device) != cudaSuccess) {
        delete ctx;
        return ALF_ERR_CUDA;
    }
    if (prop.major != 10 || prop.minor != 3) {
        // the kernels are built for sm_103a only
        delete ctx;
        return ALF_ERR_CUDA;
    }
    ctx->device = cuda_device;
    ctx->nsm = prop.multiProcessorCount;
    ctx->cc_major = prop.major;
    ctx->cc_minor = prop.minor;
    if (cudaMalloc((void**)&ctx->d_scratch_mat, sizeof(MatD)) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_scratch_env, sizeof(double) * ALF_ENV_N) != cudaSuccess) {
        dfree(ctx->d_scratch_mat);
        delete ctx;
        return ALF_ERR_OOM;
    }
    *out = ctx;
    return ALF_OK;
}

alf_status alf_destroy(alf_ctx* ctx)
{
    if (!ctx) return ALF_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    dfree(ctx->d_scratch_mat);
    dfree(ctx->d_scratch_env);
    delete ctx;
    return ALF_OK;
}

const char* alf_last_error(const alf_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

static void plan_free(alf_plan* p)
{
    if (p->chunk_graph) cudaGraphExecDestroy(p->chunk_graph);
    for (auto& e : p->ev) cudaEventDestroy(e);
    dfree(p->d_fields);
    dfree(p->d_order);
    dfree(p->d_adj_head);
    dfree(p->d_hier);
    dfree(p->d_hier_head);
    dfree(p->d_adj_nodes);
    dfree(p->d_list0);
    dfree(p->d_list1);
    dfree(p->d_elist);
    dfree(p->d_efield);
    dfree(p->d_oldv);
    dfree(p->d_newv);
    dfree(p->d_bitmap);
    dfree(p->d_bm_off);
    dfree(p->d_cnt);
    dfree(p->d_ecnt);
    dfree(p->d_eoff);
    dfree(p->d_rounds);
    dfree(p->d_flim);
    dfree(p->d_pending);
    if (p->h_pending) cudaFreeHost(p->h_pending);
    dfree(p->d_map);
    dfree(p->d_region_mat);
    dfree(p->d_mats);
    dfree(p->d_env);
    dfree(p->d_h);
    dfree(p->d_rec);
    dfree(p->d_regions);
    dfree(p->d_regions_rays);
    dfree(p->d_vtab);
    dfree(p->d_vtab64);
    dfree(p->d_regions64);
    dfree(p->d_q);
    dfree(p->d_ray_error);
    dfree(p->d_ray_blocks);
    dfree(p->d_frozen);
    if (p->h_q) cudaFreeHost(p->h_q);
}

alf_status alf_plan_create(alf_ctx* ctx, const alf_geometry* g, const alf_options* opt_in, alf_plan** out)
{
    if (!ctx) return ALF_ERR_INVALID_ARG;
    if (!g || !out) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_plan_create: null geometry or output pointer");
    *out = nullptr;
    alf_options opt;
    if (opt_in) opt = *opt_in;
    else alf_default_options(&opt);
    // ---- options
    if (opt.precision != ALF_FP32 && opt.precision != ALF_FP64)
        return fail(ctx, ALF_ERR_INVALID_ARG, "precision must be ALF_FP32 or ALF_FP64");
    if (opt.group_model != ALF_GROUP_PAPER && opt.group_model != ALF_GROUP_EXACT)
        return fail(ctx, ALF_ERR_INVALID_ARG, "unknown group_model %d", opt.group_model);
    if (opt.init_mode == ALF_INIT_RADIUS) {
        if (opt.init_radius < 0 || opt.init_radius > 8)
            return fail(ctx, ALF_ERR_INVALID_ARG, "init_radius must be in 0..8");
    } else if (opt.init_mode == ALF_INIT_HIERARCHY) {
        if (opt.n_levels < 1 || opt.n_levels > 4) return fail(ctx, ALF_ERR_INVALID_ARG, "n_levels must be in 1..4");
        for (int l = 0; l < opt.n_levels; ++l) {
            const int d = opt.level_density[l], r = opt.level_radius[l];
            if (d < 3 || d % 2 == 0 || (l > 0 && (opt.level_density[l - 1] % d != 0 || d >= opt.level_density[l - 1])))
                return fail(ctx, ALF_ERR_INVALID_ARG, "level densities must be odd, >= 3, each dividing the previous");
            if (r < 1 || r > 16 || (l > 0 && r <= opt.level_radius[l - 1]))
                return fail(ctx, ALF_ERR_INVALID_ARG, "level radii must increase within 1..16");
        }
    } else {
        return fail(ctx, ALF_ERR_INVALID_ARG, "unknown init_mode %d", opt.init_mode);
    }
    if (opt.sweep < 0 || opt.sweep > 4) return fail(ctx, ALF_ERR_INVALID_ARG, "sweep must be 0, 1, 2, 3 or 4");
    if (opt.ray_family < 0 || opt.ray_family > 5) return fail(ctx, ALF_ERR_INVALID_ARG, "ray_family must be in 0..5");
    if (opt.velocity_table != 0 && opt.velocity_table != 1)
        return fail(ctx, ALF_ERR_INVALID_ARG, "velocity_table must be 0 or 1");
    if (opt.cta_threads != 0 && opt.cta_threads != 64 && opt.cta_threads != 128 && opt.cta_threads != 256 &&
        opt.cta_threads != 512)
        return fail(ctx, ALF_ERR_INVALID_ARG, "cta_threads must be 0, 64, 128, 256 or 512");
    if (opt.cta_cluster != 0 && opt.cta_cluster != 1 && opt.cta_cluster != 2 && opt.cta_cluster != 4 &&
        opt.cta_cluster != 8)
        return fail(ctx, ALF_ERR_INVALID_ARG, "cta_cluster must be 0, 1, 2, 4 or 8");
    if (opt.cta_cluster > 1 && opt.cta_threads != 0 && opt.cta_threads != 512)
        return fail(ctx, ALF_ERR_INVALID_ARG, "cta_cluster > 1 needs cta_threads 512 (or 0)");
    if (opt.max_rounds < 1) return fail(ctx, ALF_ERR_INVALID_ARG, "max_rounds must be >= 1");
    if (opt.plane_step < 1 || opt.plane_step > 16 || opt.ray_halfwidth < 1 || opt.ray_halfwidth > 16 ||
        !(opt.stop_radius > 0.0) || opt.max_ray_points < 2 || opt.max_ray_points > (1 << 20))
        return fail(ctx, ALF_ERR_INVALID_ARG, "ray options out of range");
    if (opt.wave_mode < 0 || opt.wave_mode > 2) return fail(ctx, ALF_ERR_INVALID_ARG, "wave_mode must be 0, 1 or 2");
    if (opt.subgrid == 0) opt.subgrid = 1;  // a zeroed options struct means no refinement
    if (opt.subgrid < 1 || opt.subgrid > 21 || opt.subgrid % 2 == 0)
        return fail(ctx, ALF_ERR_INVALID_ARG, "subgrid must be an odd number in 1..21");
    const alf_options opt_caller = opt;
    const int sg = opt.subgrid;
    // lengths given in original cells become fine cells
    opt.init_radius *= sg;
    for (int l = 0; l < 4; ++l) opt.level_radius[l] *= sg;
    opt.plane_step *= sg;
    opt.ray_halfwidth *= sg;
    opt.stop_radius *= sg;
    if (opt.init_mode == ALF_INIT_HIERARCHY)
        for (int l = 0; l < opt.n_levels; ++l) {
            const long long side = 2ll * opt.level_radius[l] * opt.level_density[l] + 1;
            if (side * side > (1 << 16))
                return fail(ctx, ALF_ERR_INVALID_ARG, "level %d grid too large (%lld^2 nodes)", l, side);
        }
    // ---- geometry
    if (g->nsamples < 1 || g->nregions < 1 || g->nregions > (1 << 28) || g->nmaterials < 1 ||
        g->nmaterials > (1 << 28) || g->nsources < 1 || g->nreceivers < 0 ||
        (long long)g->nsamples * g->nregions > (1ll << 30))
        return fail(ctx, ALF_ERR_INVALID_ARG, "geometry counts out of range");
    if (!g->nx || !g->ny || !g->h || (!g->region_map && !g->region_map32) ||
        (!g->region_material && !g->region_material32) || !g->materials || !g->src_ij ||
        (g->nreceivers > 0 && !g->rec_ij))
        return fail(ctx, ALF_ERR_INVALID_ARG, "geometry has a null array");
    if (!g->region_map32 && g->nregions > 65536)
        return fail(ctx, ALF_ERR_INVALID_ARG, "more than 65536 regions need region_map32");
    if (!g->region_material32 && g->nmaterials > 65536)
        return fail(ctx, ALF_ERR_INVALID_ARG, "more than 65536 materials need region_material32");
    if (opt.velocity_table && g->nmaterials > 65536)
        return fail(ctx, ALF_ERR_INVALID_ARG, "velocity_table: at most 65536 materials");
    if (opt.wave_mode != 0 && g->nmaterials > 4096)
        return fail(ctx, ALF_ERR_INVALID_ARG, "shear wave modes: at most 4096 materials");
    std::vector<uint32_t> rmat32(g->nregions);
    for (int r = 0; r < g->nregions; ++r)
        rmat32[r] = g->region_material32 ? g->region_material32[r] : g->region_material[r];
    // region ids as 32-bit values (the device map's type), samples back to back
    std::vector<uint32_t> map32;
    {
        size_t total = 0;
        for (int b = 0; b < g->nsamples; ++b) {
            const long long nx = g->nx[b], ny = g->ny[b];
            if (nx < 2 || ny < 2 || nx > 16384 || ny > 16384 || nx * ny > (1ll << 28))
                return fail(ctx, ALF_ERR_INVALID_ARG, "sample %d: grid %lldx%lld out of range", b, nx, ny);
            total += (size_t)(nx * ny);
        }
        map32.resize(total);
        for (size_t k = 0; k < total; ++k) map32[k] = g->region_map32 ? g->region_map32[k] : g->region_map[k];
    }
    // global sub-grid (Sec. 4.5): every sample refined sg times, fine nodes taking the region of the nearest
    // original node (unique for odd sg), sources and receivers on the fine nodes of the original ones
    std::vector<int32_t> fnx, fny, fsrc, frec;
    std::vector<double> fh;
    std::vector<uint32_t> fmap;
    alf_geometry gfine;
    if (sg > 1) {
        size_t fine_total = 0;
        for (int b = 0; b < g->nsamples; ++b) {
            const long long nx = g->nx[b], ny = g->ny[b];
            if (nx < 2 || ny < 2 || (nx - 1) * sg + 1 > 16384 || (ny - 1) * sg + 1 > 16384 ||
                ((nx - 1) * sg + 1) * ((ny - 1) * sg + 1) > (1ll << 28))
                return fail(ctx, ALF_ERR_INVALID_ARG, "sample %d: grid %lldx%lld out of range with subgrid %d", b, nx,
                            ny, sg);
            fine_total += (size_t)((nx - 1) * sg + 1) * (size_t)((ny - 1) * sg + 1);
        }
        fmap.resize(fine_total);
        size_t off = 0, src_off = 0;
        for (int b = 0; b < g->nsamples; ++b) {
            const int nx = g->nx[b], ny = g->ny[b], nxf = (nx - 1) * sg + 1, nyf = (ny - 1) * sg + 1;
            fnx.push_back(nxf);
            fny.push_back(nyf);
            fh.push_back(g->h[b] / sg);
            for (int j = 0; j < nyf; ++j) {
                const int oj = (2 * j + sg) / (2 * sg);  // nearest original row
                for (int i = 0; i < nxf; ++i)
                    fmap[off + (size_t)j * nxf + i] = map32[src_off + (size_t)oj * nx + (2 * i + sg) / (2 * sg)];
            }
            off += (size_t)nxf * nyf;
            src_off += (size_t)nx * ny;
        }
        for (size_t k = 0; k < (size_t)g->nsamples * g->nsources * 2; ++k) fsrc.push_back(g->src_ij[k] * sg);
        for (size_t k = 0; k < (size_t)g->nsamples * g->nreceivers * 2; ++k) frec.push_back(g->rec_ij[k] * sg);
        gfine = *g;
        gfine.nx = fnx.data();
        gfine.ny = fny.data();
        gfine.h = fh.data();
        map32.swap(fmap);
        gfine.src_ij = fsrc.data();
        gfine.rec_ij = g->nreceivers > 0 ? frec.data() : nullptr;
        g = &gfine;
    }
    std::vector<MatD> mats(g->nmaterials);
    for (int m = 0; m < g->nmaterials; ++m)
        if (!material_to_matd(g->materials[m], opt.wave_mode, &mats[m]))
            return fail(ctx, ALF_ERR_NONPHYSICAL_MATERIAL, "material %d: rho <= 0, non-finite or non-positive c", m);
    for (int r = 0; r < g->nregions; ++r)
        if (rmat32[r] >= (uint32_t)g->nmaterials)
            return fail(ctx, ALF_ERR_INVALID_ARG, "region %d refers to material %u of %d", r, rmat32[r],
                        g->nmaterials);

    alf_plan* p = new (std::nothrow) alf_plan();
    if (!p) return fail(ctx, ALF_ERR_OOM, "host allocation");
    p->ctx = ctx;
    p->B = g->nsamples;
    p->S = g->nsources;
    p->Rr = g->nreceivers;
    p->R = g->nregions;
    p->nmat = g->nmaterials;
    p->nfields = p->B * p->S;
    p->box = opt.init_mode == ALF_INIT_HIERARCHY ? opt.level_radius[opt.n_levels - 1] : opt.init_radius;
    size_t map_off = 0, node_off = 0;
    std::vector<long long> map_offs(p->B);
    for (int b = 0; b < p->B; ++b) {
        const int nx = g->nx[b], ny = g->ny[b];
        if (nx < 2 || ny < 2 || nx > 16384 || ny > 16384 || (long long)nx * ny > (1ll << 28)) {
            delete p;
            return fail(ctx, ALF_ERR_INVALID_ARG, "sample %d: grid %dx%d out of range", b, nx, ny);
        }
        if (!(g->h[b] > 0.0) || !std::isfinite(g->h[b])) {
            delete p;
            return fail(ctx, ALF_ERR_INVALID_ARG, "sample %d: spacing must be > 0", b);
        }
        for (size_t k = 0; k < (size_t)nx * ny; ++k)
            if (map32[map_off + k] >= (uint32_t)g->nregions) {
                delete p;
                return fail(ctx, ALF_ERR_INVALID_ARG, "sample %d: region id %u >= nregions", b, map32[map_off + k]);
            }
        for (int s = 0; s < p->S; ++s) {
            const int si = g->src_ij[((size_t)b * p->S + s) * 2], sj = g->src_ij[((size_t)b * p->S + s) * 2 + 1];
            if (si < 0 || sj < 0 || si >= nx || sj >= ny) {
                delete p;
                return fail(ctx, ALF_ERR_OUT_OF_GRID, "sample %d source %d at (%d, %d) outside %dx%d", b, s, si, sj,
                            nx, ny);
            }
        }
        for (int r = 0; r < p->Rr; ++r) {
            const int ri = g->rec_ij[((size_t)b * p->Rr + r) * 2], rj = g->rec_ij[((size_t)b * p->Rr + r) * 2 + 1];
            if (ri < 0 || rj < 0 || ri >= nx || rj >= ny) {
                delete p;
                return fail(ctx, ALF_ERR_OUT_OF_GRID, "sample %d receiver %d at (%d, %d) outside %dx%d", b, r, ri,
                            rj, nx, ny);
            }
        }
        map_offs[b] = (long long)map_off;
        map_off += (size_t)nx * ny;
        p->max_field_nodes = std::max(p->max_field_nodes, (size_t)nx * ny);
    }
    p->total_map = map_off;
    // fastest qP speed over the materials (scan of phase angles; the group speed at the
    // same point of the wavefront is never below it, so this bounds the fastest front)
    double vmax = 0.0;
    // (a coarser scan when every node has its own material: the bound only sets the band width)
    const int nang = mats.size() > 4096 ? 36 : 180;
    for (const MatD& m : mats)
        for (int k = 0; k < nang; ++k) vmax = std::max(vmax, std::sqrt(mode_lambda_host(m, k * 3.141592653589793 / nang)));
    for (int b = 0; b < p->B; ++b)
        for (int s = 0; s < p->S; ++s) {
            FieldDesc fd{};
            fd.nx = g->nx[b];
            fd.ny = g->ny[b];
            fd.node_off = (long long)node_off;
            fd.map_off = map_offs[b];
            fd.sample = b;
            fd.si = g->src_ij[((size_t)b * p->S + s) * 2];
            fd.sj = g->src_ij[((size_t)b * p->S + s) * 2 + 1];
            fd.cell_time = g->h[b] / vmax;
            p->fields.push_back(fd);
            p->field_off.push_back(node_off);
            node_off += (size_t)fd.nx * fd.ny;
        }
    p->field_off.push_back(node_off);
    p->total_nodes = node_off;
    // field-resident sweep: the dirty bitmap of the largest field must fit in shared memory per warp
    p->warp_words = (unsigned)((p->max_field_nodes + 31) / 32);
    p->warp_grid = 0;
    if (p->max_field_nodes <= (size_t(1) << 18)) {
        const int c = fim_warp_ctas_per_sm(opt.precision, p->warp_words, opt.velocity_table != 0);
        p->warp_grid = c > 0 ? c * ctx->nsm : 0;
    }
    if (opt.sweep == 2 && p->warp_grid == 0) {
        delete p;
        return fail(ctx, ALF_ERR_UNSUPPORTED, "sweep = 2: a field of %zu nodes does not fit the field-resident sweep",
                    p->max_field_nodes);
    }
    // CTA-per-field sweep: shared bitmap when the largest field's fits in 64 KB, else global bitmaps
    p->cta_words = (unsigned)std::min<size_t>((p->max_field_nodes + 31) / 32, 16384);
    if (p->cta_words < (p->max_field_nodes + 31) / 32) p->cta_words = 0;
    // active-tile sweep: tile bitmaps in shared memory up to 16 KB, else the fields' global bitmaps
    {
        unsigned tw = 0;
        for (const auto& fd : p->fields) tw = std::max(tw, fim_tile_words(fd.nx, fd.ny));
        p->tile_words = tw <= 4096u ? tw : 0u;
        p->tile_grid = fim_tile_grid(opt.precision, p->tile_words, opt.velocity_table != 0, ctx->nsm);
    }
    if (opt.sweep == 4 && p->tile_grid == 0) {
        delete p;
        return fail(ctx, ALF_ERR_UNSUPPORTED, "sweep = 4: the active-tile kernel cannot be launched");
    }
    // default: a whole SM per field when the fields do not outnumber the SMs (FP32), and a cluster of 2, 4 or
    // 8 SMs per field when they leave that many SMs per field idle and the fields are large (>= 2^19 nodes
    // per SM of the cluster: on smaller fields a round is one evaluation's latency plus the cluster barrier,
    // and more SMs only add the cost of distributed shared memory; measured 6.8 vs 9.0 ms on 32 fields of
    // 256 x 256, 289 vs 228 ms on 64 fields of 2048 x 2048); else 8 warps per field
    p->cta_default = (opt.precision == ALF_FP32 && p->nfields <= ctx->nsm) ? 512 : 256;
    p->cluster_default = 1;
    if (p->cta_default == 512)
        for (int cs : {2, 4, 8})
            if ((long long)p->nfields * cs <= ctx->nsm && p->max_field_nodes >= ((size_t)cs << 19))
                p->cluster_default = cs;
    {
        const int cs = opt.cta_cluster ? opt.cta_cluster : (opt.cta_threads && opt.cta_threads != 512 ? 1 : p->cluster_default);
        set_cta_shape(p, opt.cta_threads ? opt.cta_threads : p->cta_default, cs, opt.precision, opt.velocity_table != 0);
    }
    p->sweep_mode = opt.sweep != 0 ? opt.sweep
                    : (p->warp_grid > 0 && p->nfields >= p->warp_grid * ALF_SWEEP_WARPS) ? 2 : 3;
    // launch shapes of the sweep: one warp per field for the per-field steps, a
    // persistent-sized grid for the flat evaluation and marking steps
    p->grid_fields = std::max(1, std::min((p->nfields + 7) / 8, ctx->nsm * 16));
    p->grid_eval = ctx->nsm * 16;
    std::vector<size_t> bm_off(p->nfields);
    size_t bm_words = 0;
    for (int f = 0; f < p->nfields; ++f) {
        bm_off[f] = bm_words;
        bm_words += ((size_t)p->fields[f].nx * p->fields[f].ny + 31) / 32;
    }
    p->bm_words = bm_words;
    p->opt = opt;
    p->opt_caller = opt_caller;

    cudaSetDevice(ctx->device);
    const size_t rsz = opt.precision == ALF_FP64 ? sizeof(RegionP<double>) : sizeof(RegionP<float>);
    const size_t fw = (size_t)frozen_words(p->box);
#define ALLOC(ptr, n)                                                   \
    do {                                                                \
        if (dalloc(&(ptr), (n)) != cudaSuccess) {                       \
            plan_free(p);                                               \
            delete p;                                                   \
            return fail(ctx, ALF_ERR_OOM, "workspace allocation " #ptr); \
        }                                                               \
    } while (0)
    ALLOC(p->d_fields, p->fields.size());
    ALLOC(p->d_order, p->fields.size());
    ALLOC(p->d_adj_head, 1);
    if (opt.init_mode == ALF_INIT_HIERARCHY) {
        size_t cap = 0;
        for (int l = 0; l < opt.n_levels; ++l) {
            const size_t side = 2 * (size_t)opt.level_radius[l] * opt.level_density[l] + 1;
            cap = std::max(cap, side * side);
        }
        p->hier_cap = cap;
        // one warp per field at a time; scratch bounded to about 2 GB
        const size_t stride = hier_scratch_bytes(opt.precision, cap);
        const size_t by_mem = std::max<size_t>(1, (size_t(2) << 30) / stride);
        p->hier_warps = (int)std::min<size_t>({(size_t)p->nfields, (size_t)ctx->nsm * 16, by_mem});
        char* hs = nullptr;
        ALLOC(hs, (size_t)p->hier_warps * stride);
        p->d_hier = hs;
        ALLOC(p->d_hier_head, 1);
    }
    ALLOC(p->d_list0, p->total_nodes);
    ALLOC(p->d_list1, p->total_nodes);
    ALLOC(p->d_elist, p->total_nodes);
    ALLOC(p->d_efield, p->total_nodes);
    {
        char* o = nullptr;
        char* n = nullptr;
        const size_t tb = opt.precision == ALF_FP64 ? 8 : 4;
        ALLOC(o, p->total_nodes * tb);
        p->d_oldv = o;
        ALLOC(n, p->total_nodes * tb);
        p->d_newv = n;
        char* l = nullptr;
        ALLOC(l, (size_t)p->nfields * tb);
        p->d_flim = l;
    }
    ALLOC(p->d_bitmap, p->bm_words);
    if (opt.keep_records) {
        char* w = nullptr;
        ALLOC(w, p->total_nodes * adj_node_bytes(opt.precision));
        p->d_adj_nodes = w;
    }
    ALLOC(p->d_bm_off, (size_t)p->nfields);
    ALLOC(p->d_cnt, 2 * (size_t)p->nfields);
    ALLOC(p->d_ecnt, (size_t)p->nfields);
    ALLOC(p->d_eoff, (size_t)p->nfields + 1);
    ALLOC(p->d_rounds, (size_t)p->nfields);
    ALLOC(p->d_pending, 1);
    ALLOC(p->d_map, p->total_map);
    ALLOC(p->d_region_mat, (size_t)p->R);
    ALLOC(p->d_mats, (size_t)p->nmat);
    if (opt.wave_mode != 0) ALLOC(p->d_env, (size_t)p->nmat * ALF_ENV_N);
    ALLOC(p->d_h, (size_t)p->B);
    ALLOC(p->d_rec, (size_t)p->B * p->Rr * 2);
    ALLOC(p->d_q, 1);
    ALLOC(p->d_ray_error, 4);
    ALLOC(p->d_ray_blocks, ((size_t)p->nfields * p->Rr + 1023) / 1024 + 1);
    ALLOC(p->d_frozen, (size_t)p->nfields * fw);
    {
        char* r1 = nullptr;
        char* r2 = nullptr;
        ALLOC(r1, (size_t)p->B * p->R * rsz);
        p->d_regions = r1;
        ALLOC(r2, (size_t)p->B * p->R * sizeof(RegionP<double>));
        p->d_regions64 = r2;
        char* r3 = nullptr;
        ALLOC(r3, (size_t)p->B * p->R * rsz);
        p->d_regions_rays = r3;
        if (opt.velocity_table) {
            char* t1 = nullptr;
            ALLOC(t1, (size_t)p->nmat * ALF_VTAB_N * (opt.precision == ALF_FP64 ? 8 : 4));
            p->d_vtab = t1;
            ALLOC(p->d_vtab64, (size_t)p->nmat * ALF_VTAB_N);
        }
    }
#undef ALLOC
    if (cudaMallocHost((void**)&p->h_q, sizeof(QueueState)) != cudaSuccess ||
        cudaMallocHost((void**)&p->h_pending, sizeof(unsigned long long)) != cudaSuccess) {
        plan_free(p);
        delete p;
        return fail(ctx, ALF_ERR_OOM, "pinned status word");
    }
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = up(p->d_fields, p->fields.data(), p->fields.size() * sizeof(FieldDesc));
    {
        // largest fields first: the field-resident sweep hands them out in this order
        std::vector<unsigned> order(p->fields.size());
        for (size_t f = 0; f < order.size(); ++f) order[f] = (unsigned)f;
        std::stable_sort(order.begin(), order.end(), [&](unsigned x, unsigned y) {
            return (long long)p->fields[x].nx * p->fields[x].ny > (long long)p->fields[y].nx * p->fields[y].ny;
        });
        if (e == cudaSuccess) e = up(p->d_order, order.data(), order.size() * sizeof(unsigned));
    }
    if (e == cudaSuccess) e = up(p->d_map, map32.data(), p->total_map * sizeof(uint32_t));
    if (e == cudaSuccess) e = up(p->d_bm_off, bm_off.data(), bm_off.size() * sizeof(size_t));
    if (e == cudaSuccess) e = up(p->d_region_mat, rmat32.data(), (size_t)p->R * sizeof(uint32_t));
    if (e == cudaSuccess) e = up(p->d_mats, mats.data(), mats.size() * sizeof(MatD));
    if (e == cudaSuccess && opt.wave_mode != 0) {
        // shear modes: every material's envelope table on the device, then the materials point at theirs
        e = launch_env_table(p->d_mats, p->nmat, p->d_env, nullptr);
        for (int m = 0; m < p->nmat; ++m) mats[m].env = p->d_env + (size_t)m * ALF_ENV_N;
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = up(p->d_mats, mats.data(), mats.size() * sizeof(MatD));
    }
    if (e == cudaSuccess && opt.velocity_table) {
        // phase speed of every material at 0..180 degrees from its axis (the qP eigenvalue of the rotated
        // Christoffel matrix, Sec. 3.2)
        std::vector<double> t64((size_t)p->nmat * ALF_VTAB_N);
        for (int m = 0; m < p->nmat; ++m)
            for (int k = 0; k < ALF_VTAB_N; ++k)
                t64[(size_t)m * ALF_VTAB_N + k] = std::sqrt(mode_lambda_host(mats[m], k * 3.141592653589793 / 180.0));
        e = up(p->d_vtab64, t64.data(), t64.size() * sizeof(double));
        if (e == cudaSuccess) {
            if (opt.precision == ALF_FP64) {
                e = up(p->d_vtab, t64.data(), t64.size() * sizeof(double));
            } else {
                std::vector<float> t32(t64.begin(), t64.end());
                e = up(p->d_vtab, t32.data(), t32.size() * sizeof(float));
            }
        }
    }
    if (e == cudaSuccess) e = up(p->d_h, g->h, (size_t)p->B * sizeof(double));
    if (e == cudaSuccess && p->Rr) e = up(p->d_rec, g->rec_ij, (size_t)p->B * p->Rr * 2 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(p->d_ray_error, 0, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        plan_free(p);
        delete p;
        return fail(ctx, ALF_ERR_CUDA, "plan upload: %s", cudaGetErrorString(e));
    }
    *out = p;
    return ALF_OK;
}

alf_status alf_plan_destroy(alf_plan* p)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    cudaSetDevice(p->ctx->device);
    cudaDeviceSynchronize();
    plan_free(p);
    delete p;
    return ALF_OK;
}

size_t alf_plan_field_offset(const alf_plan* p, int f)
{
    if (!p || f < 0 || f > p->nfields) return 0;
    return p->field_off[f];
}

int alf_plan_nfields(const alf_plan* p) { return p ? p->nfields : 0; }

alf_status alf_plan_options(const alf_plan* p, alf_options* out)
{
    if (!p || !out) return ALF_ERR_INVALID_ARG;
    // lengths as the caller gave them (original cells); the schedule and band in effect
    *out = p->opt_caller;
    out->band_cells = p->opt.band_cells;
    out->sweep = p->sweep_mode;
    out->cta_threads = p->cta_threads;
    out->cta_cluster = p->cta_cluster;
    return ALF_OK;
}

}  // extern "C"

// The forward solve; with max_rel / n_flips also the FP64 check of its fields (alf_solve_check64), fused into
// the CTA sweep where that kernel can run it, else launched after the solve.
static alf_status solve_impl(alf_plan* p, const double* theta, void* times, void* rec_times, uint8_t* records,
                             double* max_rel, int32_t* n_flips, cudaStream_t st)
{
    alf_ctx* ctx = p->ctx;
    const int prec = p->opt.precision;
    const int gm = p->opt.group_model;
    const bool fused = max_rel && p->sweep_mode == 3 && !p->opt.time_kernels &&
                       fim_cta_can_check(prec, p->opt.velocity_table, p->cta_cluster);
    if (max_rel) {
        ALF_CUDA(ctx, launch_prep_regions(ALF_FP64, p->d_mats, p->d_region_mat, theta, p->d_h, p->B, p->R, gm,
                                          p->d_regions64, st, p->d_vtab64));
    }
    ALF_CUDA(ctx, launch_prep_regions(prec, p->d_mats, p->d_region_mat, theta, p->d_h, p->B, p->R, gm, p->d_regions, st,
                                      p->d_vtab));
    ALF_CUDA(ctx, launch_fill_inf(prec, times, p->total_nodes, st));
    if (records) ALF_CUDA(ctx, cudaMemsetAsync(records, 255, p->total_nodes, st));
    ALF_CUDA(ctx, cudaMemsetAsync(p->d_frozen, 0, sizeof(unsigned) * (size_t)p->nfields * frozen_words(p->box), st));
    ALF_CUDA(ctx, cudaMemsetAsync(p->d_q, 0, sizeof(QueueState), st));
    if (p->opt.init_mode == ALF_INIT_HIERARCHY) {
        ALF_CUDA(ctx, cudaMemsetAsync(p->d_hier_head, 0, sizeof(unsigned), st));
        HierLaunch h;
        h.times = times;
        h.fields = p->d_fields;
        h.nfields = p->nfields;
        h.region_map = p->d_map;
        h.region_mat = p->d_region_mat;
        h.mats = p->d_mats;
        h.regions = p->d_regions;
        h.theta = theta;
        h.h = p->d_h;
        h.nregions = p->R;
        h.group_model = gm;
        h.nlev = p->opt.n_levels;
        for (int l = 0; l < 4; ++l) {
            h.dens[l] = p->opt.level_density[l];
            h.rad[l] = p->opt.level_radius[l];
        }
        h.box = p->box;
        h.frozen_bits = p->d_frozen;
        h.level_cap = p->hier_cap;
        h.scratch = p->d_hier;
        h.scratch_stride = hier_scratch_bytes(prec, p->hier_cap);
        h.nwarps = p->hier_warps;
        h.head = p->d_hier_head;
        h.q = p->d_q;
        h.band_cells = p->opt.band_cells;
        h.max_rounds_per_node = (unsigned)p->opt.max_rounds;
        h.vtable = p->opt.velocity_table;
        ALF_CUDA(ctx, launch_init_hierarchy(prec, h, st));
    } else {
        ALF_CUDA(ctx, launch_init_radius(prec, times, p->d_fields, p->nfields, p->d_map, p->d_region_mat, p->d_mats,
                                         theta, p->d_h, p->R, p->opt.init_radius, gm, p->d_frozen, p->box, st));
    }
    FimLaunch a;
    a.times = times;
    a.fields = p->d_fields;
    a.nfields = p->nfields;
    a.region_map = p->d_map;
    a.regions = p->d_regions;
    a.nregions = p->R;
    a.box = p->box;
    a.list[0] = p->d_list0;
    a.list[1] = p->d_list1;
    a.elist = p->d_elist;
    a.bitmap = p->d_bitmap;
    a.bm_off = p->d_bm_off;
    a.cnt = p->d_cnt;
    a.ecnt = p->d_ecnt;
    a.eoff = p->d_eoff;
    a.efield = p->d_efield;
    a.oldv = p->d_oldv;
    a.newv = p->d_newv;
    a.rounds = p->d_rounds;
    a.flim = p->d_flim;
    a.max_rounds_per_node = (unsigned)p->opt.max_rounds;
    a.band_cells = p->opt.band_cells;
    a.q = p->d_q;
    a.records = records;
    a.vtable = p->opt.velocity_table;
    if (fused) {
        ALF_CUDA(ctx, cudaMemsetAsync(max_rel, 0, sizeof(double) * p->nfields, st));
        ALF_CUDA(ctx, cudaMemsetAsync(n_flips, 0, sizeof(int32_t) * p->nfields, st));
        a.regions64 = p->d_regions64;
        a.frozen_bits = p->d_frozen;
        a.max_rel = max_rel;
        a.n_flips = n_flips;
    }
    if (p->sweep_mode >= 2) {
        // field-resident sweep: the whole fixed-point iteration in one launch
        const bool timing = p->opt.time_kernels != 0;
        if (timing && p->ev.size() < 2) {
            p->ev.resize(2);
            for (auto& e : p->ev) ALF_CUDA(ctx, cudaEventCreate(&e));
        }
        if (timing) ALF_CUDA(ctx, cudaEventRecord(p->ev[0], st));
        if (p->sweep_mode == 2) ALF_CUDA(ctx, launch_fim_warp(prec, a, p->d_order, p->warp_words, p->warp_grid, st));
        else if (p->sweep_mode == 4)
            ALF_CUDA(ctx, launch_fim_tile(prec, a, p->d_order, p->tile_words, p->tile_grid, st));
        else
            ALF_CUDA(ctx, launch_fim_cta(prec, a, p->d_order, p->cta_words, p->cta_grid, p->cta_threads, p->cta_cluster,
                                         st, fused));
        if (timing) {
            ALF_CUDA(ctx, cudaEventRecord(p->ev[1], st));
            ALF_CUDA(ctx, cudaEventSynchronize(p->ev[1]));
            float ms = 0.f;
            ALF_CUDA(ctx, cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]));
            p->eval_ms = ms;
            p->eval_launches = 1;
        }
        p->sweep_rounds = 0;  // per-field counts: alf_plan_stats reads the largest
    } else {
        ALF_CUDA(ctx, launch_fim_init(prec, a, p->grid_fields, st));
        const alf_status rc = run_sweep(p, a, st);
        if (rc != ALF_OK) return rc;
    }
    ALF_CUDA(ctx, launch_finalize(prec, times, p->d_fields, p->nfields, p->box, p->d_rec, p->S, p->Rr, rec_times,
                                  records, st));
    if (max_rel && !fused)
        ALF_CUDA(ctx, launch_check64(prec, times, p->d_fields, p->nfields, p->d_map, p->d_regions64, p->R, records,
                                     p->d_frozen, p->box, max_rel, n_flips, ctx->nsm * ALF_CHECK_CTAS_PER_SM, st,
                                     p->opt.velocity_table));
    return ALF_OK;
}

extern "C" {

alf_status alf_solve(alf_plan* p, const double* theta, void* times, void* rec_times, uint8_t* records, void* stream)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    if (!theta || !times) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_solve: null theta or times");
    if (rec_times && p->Rr == 0) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_solve: plan has no receivers");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    return solve_impl(p, theta, times, rec_times, records, nullptr, nullptr, as_stream(stream));
}

alf_status alf_solve_check64(alf_plan* p, const double* theta, void* times, void* rec_times, uint8_t* records,
                             double* max_rel, int32_t* n_flips, void* stream)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    if (!theta || !times || !max_rel || !n_flips)
        return fail(ctx, ALF_ERR_INVALID_ARG, "alf_solve_check64: null theta, times, max_rel or n_flips");
    if (rec_times && p->Rr == 0) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_solve_check64: plan has no receivers");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    return solve_impl(p, theta, times, rec_times, records, max_rel, n_flips, as_stream(stream));
}

alf_status alf_check64(alf_plan* p, const double* theta, const void* times, const uint8_t* records, double* max_rel,
                       int32_t* n_flips, void* stream)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    if (!theta || !times || !max_rel || !n_flips) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_check64: null pointer");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = as_stream(stream);
    ALF_CUDA(ctx, launch_prep_regions(ALF_FP64, p->d_mats, p->d_region_mat, theta, p->d_h, p->B, p->R,
                                      p->opt.group_model, p->d_regions64, st, p->d_vtab64));
    ALF_CUDA(ctx, launch_check64(p->opt.precision, times, p->d_fields, p->nfields, p->d_map, p->d_regions64, p->R,
                                 records, p->d_frozen, p->box, max_rel, n_flips, ctx->nsm * ALF_CHECK_CTAS_PER_SM, st,
                                 p->opt.velocity_table));
    return ALF_OK;
}

alf_status alf_check64_nodes(alf_plan* p, const double* theta, const void* times, const uint8_t* records,
                             double* check_times, uint8_t* check_records, double* max_rel, int32_t* n_flips,
                             void* stream)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    if (!theta || !times || !max_rel || !n_flips || (!check_times && !check_records))
        return fail(ctx, ALF_ERR_INVALID_ARG, "alf_check64_nodes: null pointer");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = as_stream(stream);
    ALF_CUDA(ctx, launch_prep_regions(ALF_FP64, p->d_mats, p->d_region_mat, theta, p->d_h, p->B, p->R,
                                      p->opt.group_model, p->d_regions64, st, p->d_vtab64));
    ALF_CUDA(ctx, launch_check64(p->opt.precision, times, p->d_fields, p->nfields, p->d_map, p->d_regions64, p->R,
                                 records, p->d_frozen, p->box, max_rel, n_flips, ctx->nsm * ALF_CHECK_CTAS_PER_SM, st,
                                 p->opt.velocity_table, check_times, check_records));
    return ALF_OK;
}

alf_status alf_trace_rays(alf_plan* p, const double* theta, const void* times, void* ray_pts, int32_t* ray_npts,
                          void* ray_time, int32_t* ray_status, void* stream)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    if (!theta || !times || !ray_pts || !ray_npts)
        return fail(ctx, ALF_ERR_INVALID_ARG, "alf_trace_rays: null theta, times, ray_pts or ray_npts");
    if (p->Rr == 0) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_trace_rays: plan has no receivers");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = as_stream(stream);
    // rays keep their own region constants, so that they can run beside alf_check64 and alf_backward
    ALF_CUDA(ctx, launch_prep_regions(p->opt.precision, p->d_mats, p->d_region_mat, theta, p->d_h, p->B, p->R,
                                      p->opt.group_model, p->d_regions_rays, st));
    RayLaunch a;
    a.times = times;
    a.fields = p->d_fields;
    a.nfields = p->nfields;
    a.region_map = p->d_map;
    a.region_mat = p->d_region_mat;
    a.mats = p->d_mats;
    a.regions = p->d_regions_rays;
    a.theta = theta;
    a.nregions = p->R;
    a.rec_ij = p->d_rec;
    a.nsrc = p->S;
    a.nrec = p->Rr;
    a.group_model = p->opt.group_model;
    a.plane_step = p->opt.plane_step;
    a.family = p->opt.ray_family - 1;
    a.halfwidth = p->opt.ray_halfwidth;
    a.max_pts = p->opt.max_ray_points;
    a.stop_radius = p->opt.stop_radius;
    a.pts = ray_pts;
    a.npts = ray_npts;
    a.ray_time = ray_time;
    a.ray_status = ray_status;
    a.error = p->d_ray_error;
    a.h_of_sample = p->d_h;
    ALF_CUDA(ctx, launch_rays(p->opt.precision, a, st));
    return ALF_OK;
}

alf_status alf_pack_rays(alf_plan* p, const void* ray_pts, const int32_t* ray_npts, void* packed_pts,
                         int64_t* offsets, void* stream)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    if (!ray_pts || !ray_npts || !packed_pts || !offsets)
        return fail(ctx, ALF_ERR_INVALID_ARG, "alf_pack_rays: null ray_pts, ray_npts, packed_pts or offsets");
    if (p->Rr == 0) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_pack_rays: plan has no receivers");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    ALF_CUDA(ctx, launch_pack_rays(p->opt.precision, ray_pts, ray_npts, (long long)p->nfields * p->Rr,
                                   p->opt.max_ray_points, p->d_ray_blocks, packed_pts, (long long*)offsets,
                                   ctx->nsm * 16, as_stream(stream)));
    return ALF_OK;
}

alf_status alf_ray_gradient(alf_plan* p, const double* theta, const void* ray_pts, const int32_t* ray_npts,
                            const void* dL_dray, double* dL_dtheta, void* stream)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    if (!theta || !ray_pts || !ray_npts || !dL_dray || !dL_dtheta)
        return fail(ctx, ALF_ERR_INVALID_ARG, "alf_ray_gradient: null pointer");
    if (p->Rr == 0) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_ray_gradient: plan has no receivers");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = as_stream(stream);
    RayLaunch a{};
    a.fields = p->d_fields;
    a.nfields = p->nfields;
    a.region_map = p->d_map;
    a.region_mat = p->d_region_mat;
    a.mats = p->d_mats;
    a.theta = theta;
    a.nregions = p->R;
    a.nsrc = p->S;
    a.nrec = p->Rr;
    a.group_model = p->opt.group_model;
    a.max_pts = p->opt.max_ray_points;
    a.pts = const_cast<void*>(ray_pts);
    a.npts = const_cast<int32_t*>(ray_npts);
    a.h_of_sample = p->d_h;
    ALF_CUDA(ctx, launch_ray_gradient(p->opt.precision, a, dL_dray, dL_dtheta, p->B, st));
    return ALF_OK;
}

alf_status alf_backward(alf_plan* p, const double* theta, const void* times, const uint8_t* records,
                        const void* dL_drec, double* dL_dtheta, void* stream)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    if (!theta || !times || !records || !dL_drec || !dL_dtheta)
        return fail(ctx, ALF_ERR_INVALID_ARG, "alf_backward: null pointer");
    if (!p->opt.keep_records || !p->d_adj_nodes)
        return fail(ctx, ALF_ERR_INVALID_ARG, "alf_backward: the plan was created without keep_records");
    if (p->opt.init_mode != ALF_INIT_RADIUS)
        return fail(ctx, ALF_ERR_UNSUPPORTED, "alf_backward: only the straight-ray initialisation is differentiated");
    if (p->opt.velocity_table)
        return fail(ctx, ALF_ERR_UNSUPPORTED, "alf_backward: the velocity-table update is not differentiated");
    if (p->Rr == 0) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_backward: plan has no receivers");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = as_stream(stream);
    const int prec = p->opt.precision;
    ALF_CUDA(ctx, launch_prep_regions(prec, p->d_mats, p->d_region_mat, theta, p->d_h, p->B, p->R, p->opt.group_model,
                                      p->d_regions, st));
    AdjLaunch a;
    a.times = times;
    a.fields = p->d_fields;
    a.nfields = p->nfields;
    a.nsamples = p->B;
    a.nrec = p->Rr;
    a.total_nodes = p->total_nodes;
    a.region_map = p->d_map;
    a.region_mat = p->d_region_mat;
    a.mats = p->d_mats;
    a.regions = p->d_regions;
    a.theta = theta;
    a.h = p->d_h;
    a.nregions = p->R;
    a.box = p->box;
    a.group_model = p->opt.group_model;
    a.frozen_bits = p->d_frozen;
    a.records = records;
    a.rec_ij = p->d_rec;
    a.nodes = p->d_adj_nodes;
    a.list[0] = p->d_list0;
    a.list[1] = p->d_list1;
    a.cnt = p->d_cnt;
    a.eoff = p->d_eoff;
    long long mx = 0;
    for (const FieldDesc& fd : p->fields) mx = std::max(mx, (long long)fd.nx * fd.ny);
    a.max_rounds = (unsigned)std::min<long long>(mx + 64, 0x7fffffffll);
    a.order = p->d_order;
    a.head = p->d_adj_head;
    // One warp per field when the forward ran one (sweep 2) or when the fields fill the GPU's 16 adjoint
    // warps per SM; else the lockstep rounds, which spread a few large fields over every SM.  The schedule
    // is independent of how the forward reached its fixed point: both read the same records.
    // 2 CTAs of 8 warps per SM: fewer fields in flight keep more of their fronts in L2 (measured
    // 129 / 116 / 114 ms for 8 / 4 / 2 CTAs per SM on the 512 x 32 weld batch)
    const bool adj_warp = p->sweep_mode == 2 || p->nfields >= p->ctx->nsm * 16;
    a.warp_grid = adj_warp ? p->ctx->nsm * 2 : 0;
    a.q = p->d_q;
    ALF_CUDA(ctx, launch_adjoint(prec, a, dL_drec, dL_dtheta, p->d_pending, p->h_pending, p->grid_eval, st));
    return ALF_OK;
}

alf_status alf_sync_status(alf_plan* p, void* stream, int32_t* worst)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = as_stream(stream);
    ALF_CUDA(ctx, cudaMemcpyAsync(p->h_q, p->d_q, sizeof(QueueState), cudaMemcpyDeviceToHost, st));
    unsigned ray_err = 0;
    ALF_CUDA(ctx, cudaStreamSynchronize(st));
    ALF_CUDA(ctx, cudaMemcpy(&ray_err, p->d_ray_error, sizeof(unsigned), cudaMemcpyDeviceToHost));
    unsigned code = p->h_q->error;
    if (code == 0) code = ray_err;
    ALF_CUDA(ctx, cudaMemset(p->d_ray_error, 0, sizeof(unsigned)));
    p->h_q->error = 0;
    ALF_CUDA(ctx, cudaMemcpy(&p->d_q->error, &p->h_q->error, sizeof(unsigned), cudaMemcpyHostToDevice));
    if (worst) *worst = (int32_t)code;
    if (code != 0)
        return fail(ctx, (alf_status)code, "device status %u (node evaluations %llu)", code,
                    (unsigned long long)p->h_q->visits);
    return ALF_OK;
}

alf_status alf_plan_stats(alf_plan* p, void* stream, alf_stats* out)
{
    if (!p || !out) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = as_stream(stream);
    ALF_CUDA(ctx, cudaMemcpyAsync(p->h_q, p->d_q, sizeof(QueueState), cudaMemcpyDeviceToHost, st));
    ALF_CUDA(ctx, cudaStreamSynchronize(st));
    out->node_evaluations = p->h_q->visits;
    out->rounds = p->sweep_mode != 1 ? p->h_q->rounds : p->sweep_rounds;
    out->nodes = (uint64_t)p->total_nodes;
    out->eval_launches = p->eval_launches;
    out->eval_ms = p->eval_ms;
    out->kernel_launches = launches_so_far();
    out->dirty_entries = p->h_q->dirty;
    return ALF_OK;
}

alf_status alf_plan_autotune(alf_plan* p, const double* theta, void* times, uint8_t* records, void* stream)
{
    if (!p) return ALF_ERR_INVALID_ARG;
    alf_ctx* ctx = p->ctx;
    if (!theta || !times) return fail(ctx, ALF_ERR_INVALID_ARG, "alf_plan_autotune: null theta or times");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = as_stream(stream);
    // candidates: (schedule, band, evaluation block); a schedule fixed by the options is kept
    struct Cand {
        int mode;
        double band;
        int block;
        int cluster;
    };
    std::vector<Cand> cands;
    const bool try1 = p->opt.sweep == 0 || p->opt.sweep == 1;
    const bool try2 = (p->opt.sweep == 0 || p->opt.sweep == 2) && p->warp_grid > 0;
    // (block: the evaluation block of the lockstep rounds, the threads of one field's CTA for sweep 3)
    if (try1)
        for (double band : {2.0, 3.0, 4.0, 6.0})
            for (int blk : {128, 256}) cands.push_back({1, band, blk, 1});
    // bands of the field-resident schedules: measured optima lie between 1.5 and 2.5 cells on weld media
    if (try2)
        for (double band : {1.0, 1.5, 2.0, 2.5, 3.0, 4.0}) cands.push_back({2, band, p->eval_block, 1});
    if (p->opt.sweep == 0 || p->opt.sweep == 3)
        for (double band : {1.0, 1.5, 2.0, 2.5, 3.0}) {
            if (p->opt.cta_cluster <= 1)
                for (int nt : {64, 128, 256, 512})
                    if (p->opt.cta_threads == 0 || p->opt.cta_threads == nt) cands.push_back({3, band, nt, 1});
            // clusters only where fields leave SMs idle
            for (int cs : {2, 4, 8})
                if ((p->opt.cta_cluster == 0 || p->opt.cta_cluster == cs) &&
                    (p->opt.cta_threads == 0 || p->opt.cta_threads == 512) && (long long)p->nfields * cs <= 2 * p->ctx->nsm)
                    cands.push_back({3, band, 512, cs});
        }
    double best_ms = 1e30, best_band = p->opt.band_cells;
    const int eval_block0 = p->eval_block;
    int best_block = p->sweep_mode == 3 ? p->cta_threads : p->eval_block, best_mode = p->sweep_mode;
    int best_cluster = p->cta_cluster;
    // the plan's settings before tuning, put back if a candidate fails
    const double band0 = p->opt.band_cells;
    const int mode0 = p->sweep_mode, threads0 = p->cta_threads, cluster0 = p->cta_cluster;
    cudaEvent_t e0, e1;
    ALF_CUDA(ctx, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, ALF_ERR_CUDA, "alf_plan_autotune: cudaEventCreate failed");
    }
    const int keep_timing = p->opt.time_kernels;
    p->opt.time_kernels = 0;
    // one candidate: a warm-up solve (graph capture), then the faster of two timed solves (the candidates
    // often differ by a few %)
    auto time_candidate = [&](const Cand& c, float* ms) -> alf_status {
        p->opt.band_cells = c.band;
        p->eval_block = c.mode == 1 ? c.block : eval_block0;
        if (c.mode == 3) set_cta_shape(p, c.block, c.cluster, p->opt.precision, p->opt.velocity_table != 0);
        p->sweep_mode = c.mode;
        if (p->chunk_graph) {
            cudaGraphExecDestroy(p->chunk_graph);
            p->chunk_graph = nullptr;
        }
        alf_status rc = alf_solve(p, theta, times, nullptr, records, stream);
        if (rc != ALF_OK) return rc;
        *ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            ALF_CUDA(ctx, cudaEventRecord(e0, st));
            rc = alf_solve(p, theta, times, nullptr, records, stream);
            if (rc != ALF_OK) return rc;
            ALF_CUDA(ctx, cudaEventRecord(e1, st));
            ALF_CUDA(ctx, cudaEventSynchronize(e1));
            float m = 0.f;
            ALF_CUDA(ctx, cudaEventElapsedTime(&m, e0, e1));
            *ms = std::min(*ms, m);
        }
        return ALF_OK;
    };
    alf_status status = ALF_OK;
    for (const Cand& c : cands) {
        float ms = 0.f;
        status = time_candidate(c, &ms);
        if (status != ALF_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best_band = c.band;
            best_block = c.block;
            best_mode = c.mode;
            best_cluster = c.cluster;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->opt.time_kernels = keep_timing;
    if (p->chunk_graph) {
        cudaGraphExecDestroy(p->chunk_graph);
        p->chunk_graph = nullptr;
    }
    if (status != ALF_OK) {
        p->opt.band_cells = band0;
        p->eval_block = eval_block0;
        set_cta_shape(p, threads0, cluster0, p->opt.precision, p->opt.velocity_table != 0);
        p->sweep_mode = mode0;
        return status;
    }
    p->opt.band_cells = best_band;
    p->eval_block = best_mode == 1 ? best_block : eval_block0;
    if (best_mode == 3)
        set_cta_shape(p, best_block, best_cluster, p->opt.precision, p->opt.velocity_table != 0);
    else
        set_cta_shape(p, p->opt.cta_threads ? p->opt.cta_threads : p->cta_default,
                      p->opt.cta_cluster ? p->opt.cta_cluster : p->cluster_default, p->opt.precision,
                      p->opt.velocity_table != 0);
    p->sweep_mode = best_mode;
    return ALF_OK;
}

alf_status alf_eval_velocity(alf_ctx* ctx, const alf_material* mat, int kind, int group_model, int precision,
                             const double* angles, double* out, int n, void* stream)
{
    if (!ctx) return ALF_ERR_INVALID_ARG;
    if (!mat || !angles || !out || n < 0 || kind < 0 || kind > 5 ||
        (group_model != ALF_GROUP_PAPER && group_model != ALF_GROUP_EXACT) ||
        (precision != ALF_FP32 && precision != ALF_FP64))
        return fail(ctx, ALF_ERR_INVALID_ARG, "alf_eval_velocity: bad argument");
    const int mode = kind / 2;
    MatD m;
    if (!material_to_matd(*mat, mode, &m)) return fail(ctx, ALF_ERR_NONPHYSICAL_MATERIAL, "alf_eval_velocity: material");
    ALF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = as_stream(stream);
    ALF_CUDA(ctx, cudaMemcpyAsync(ctx->d_scratch_mat, &m, sizeof(MatD), cudaMemcpyHostToDevice, st));
    if (mode != 0) {
        // the shear modes' group speeds come from the material's envelope table
        ALF_CUDA(ctx, launch_env_table(ctx->d_scratch_mat, 1, ctx->d_scratch_env, st));
        m.env = ctx->d_scratch_env;
        ALF_CUDA(ctx, cudaMemcpyAsync(ctx->d_scratch_mat, &m, sizeof(MatD), cudaMemcpyHostToDevice, st));
    }
    ALF_CUDA(ctx, cudaStreamSynchronize(st));
    if (n == 0) return ALF_OK;
    ALF_CUDA(ctx, launch_eval_velocity(ctx->d_scratch_mat, kind % 2, group_model, precision, angles, out, n, st));
    return ALF_OK;
}

}  // extern "C"
