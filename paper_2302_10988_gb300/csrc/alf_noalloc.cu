// alf_noalloc.cu -- a forward solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// entirely owned by another allocator (a framework's caching pool sized to
// the whole GPU, or a fixed arena handed out at start-up), and latency-bound
// loops for which cudaMalloc/cudaFree are off limits because they can
// synchronise the whole device and take unbounded time.  alf_solve_field_noalloc
// serves them: it solves one field with the same kernels as alf_solve, but
// every workspace it needs lives in the file-scope device array below, which
// the CUDA runtime creates when the library is loaded (every GPU that loads
// the library holds it until the process exits).
//
// Host code cannot use the array's name as a device address (on the host it
// only names a stand-in symbol), so the device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device; that first call should therefore come before any
// stream capture.  All calls share the array and it keeps the last call's
// contents: everything that must start at zero is cleared by each call, and
// calls whose work overlaps on the GPU (on different streams, or from
// different host threads) race on it.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "alf_internal.h"

namespace alf {
namespace {

// Limits of the allocation-free solve (the array is about 8 MB).
constexpr int kNoAllocMaxNodes = 512 * 512;
constexpr int kNoAllocMaxRegions = 1024;
constexpr int kNoAllocMaxMaterials = 64;
constexpr int kNoAllocMaxInitRadius = 8;

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Layout of the scratch array (byte offsets).
constexpr size_t kOffQ = 0;
constexpr size_t kOffField = align256(kOffQ + sizeof(QueueState));
constexpr size_t kOffMats = align256(kOffField + sizeof(FieldDesc));
constexpr size_t kOffRegions = align256(kOffMats + sizeof(MatD) * kNoAllocMaxMaterials);
constexpr size_t kOffH = align256(kOffRegions + sizeof(RegionP<float>) * kNoAllocMaxRegions);
constexpr size_t kOffFrozen = align256(kOffH + sizeof(double));
constexpr size_t kFrozenWords = ((2 * kNoAllocMaxInitRadius + 1) * (2 * kNoAllocMaxInitRadius + 1) + 31) / 32;
constexpr size_t kOffCounters = align256(kOffFrozen + sizeof(unsigned) * kFrozenWords);
// counters: cnt[2], ecnt, eoff[2], rounds, bm_off (size_t), pending (u64), flim (float)
constexpr size_t kOffList0 = align256(kOffCounters + 128);
constexpr size_t kOffList1 = align256(kOffList0 + sizeof(unsigned) * kNoAllocMaxNodes);
constexpr size_t kOffElist = align256(kOffList1 + sizeof(unsigned) * kNoAllocMaxNodes);
constexpr size_t kOffEfield = align256(kOffElist + sizeof(unsigned) * kNoAllocMaxNodes);
constexpr size_t kOffOld = align256(kOffEfield + sizeof(unsigned) * kNoAllocMaxNodes);
constexpr size_t kOffNew = align256(kOffOld + sizeof(float) * kNoAllocMaxNodes);
constexpr size_t kOffBitmap = align256(kOffNew + sizeof(float) * kNoAllocMaxNodes);
constexpr size_t kOffMap32 = align256(kOffBitmap + sizeof(unsigned) * ((kNoAllocMaxNodes + 31) / 32));
constexpr size_t kOffRmat32 = align256(kOffMap32 + sizeof(uint32_t) * kNoAllocMaxNodes);
constexpr size_t kScratchBytes = align256(kOffRmat32 + sizeof(uint32_t) * kNoAllocMaxRegions);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_addr_mu;
void* g_addr[64] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = (unsigned char*)g_addr[dev];
    return cudaSuccess;
}

// Copies the caller's 16-bit region map and region->material table into the 32-bit ones the kernels read, and
// flags (word *bad = 1) a region id >= nregions or a material id >= nmaterials: the kernels index the region
// constants and the material table with them.
__global__ void check_ids_kernel(const uint16_t* region_map, int n, const uint16_t* region_material, int nregions,
                                 int nmaterials, uint32_t* map32, uint32_t* rmat32, unsigned* bad)
{
    bool out = false;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t r = region_map[k];
        map32[k] = r;
        out |= r >= (uint32_t)nregions;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nregions; k += gridDim.x * blockDim.x) {
        const uint32_t m = region_material[k];
        rmat32[k] = m;
        out |= m >= (uint32_t)nmaterials;
    }
    if (out) *bad = 1u;
}

alf_status nfail(char* err, size_t len, alf_status code, const char* msg)
{
    if (err && len) {
        std::strncpy(err, msg, len - 1);
        err[len - 1] = '\0';
    }
    return code;
}

}  // namespace
}  // namespace alf

using namespace alf;

extern "C" alf_status alf_solve_field_noalloc(int cuda_device, const alf_material* materials, int nmaterials,
                                              const uint16_t* region_material, int nregions,
                                              const double* region_theta, const uint16_t* region_map, int nx, int ny,
                                              double h, int si, int sj, int init_radius, int group_model,
                                              int max_rounds, float* times, void* stream, char* err, size_t err_len)
{
    char msg[256];
    if (!materials || !region_material || !region_theta || !region_map || !times)
        return nfail(err, err_len, ALF_ERR_INVALID_ARG, "alf_solve_field_noalloc: null pointer");
    if (nx < 2 || ny < 2 || (long long)nx * ny > kNoAllocMaxNodes) {
        std::snprintf(msg, sizeof(msg), "alf_solve_field_noalloc: grid %dx%d exceeds the limit of %d nodes", nx, ny,
                      kNoAllocMaxNodes);
        return nfail(err, err_len, ALF_ERR_INVALID_ARG, msg);
    }
    if (nregions < 1 || nregions > kNoAllocMaxRegions || nmaterials < 1 || nmaterials > kNoAllocMaxMaterials) {
        std::snprintf(msg, sizeof(msg),
                      "alf_solve_field_noalloc: %d regions / %d materials exceed the limits %d / %d", nregions,
                      nmaterials, kNoAllocMaxRegions, kNoAllocMaxMaterials);
        return nfail(err, err_len, ALF_ERR_INVALID_ARG, msg);
    }
    if (init_radius < 0 || init_radius > kNoAllocMaxInitRadius)
        return nfail(err, err_len, ALF_ERR_INVALID_ARG, "alf_solve_field_noalloc: init_radius must be in 0..8");
    if (group_model != ALF_GROUP_PAPER && group_model != ALF_GROUP_EXACT)
        return nfail(err, err_len, ALF_ERR_INVALID_ARG, "alf_solve_field_noalloc: unknown group model");
    if (!(h > 0.0) || !std::isfinite(h))
        return nfail(err, err_len, ALF_ERR_INVALID_ARG, "alf_solve_field_noalloc: spacing must be > 0");
    if (max_rounds < 0) return nfail(err, err_len, ALF_ERR_INVALID_ARG, "alf_solve_field_noalloc: max_rounds < 0");
    if (si < 0 || sj < 0 || si >= nx || sj >= ny)
        return nfail(err, err_len, ALF_ERR_OUT_OF_GRID, "alf_solve_field_noalloc: source outside the grid");
    MatD mats[kNoAllocMaxMaterials];
    double vmax = 0.0;
    for (int m = 0; m < nmaterials; ++m) {
        const alf_material& M = materials[m];
        const double c22 = M.c[1][1], c23 = M.c[1][2], c33 = M.c[2][2], c44 = M.c[3][3], rho = M.rho;
        if (!(rho > 0.0) || !std::isfinite(rho) || !std::isfinite(c23) || !(c22 > 0.0) || !(c33 > 0.0) ||
            !(c44 > 0.0) || !std::isfinite(c22) || !std::isfinite(c33) || !std::isfinite(c44) ||
            !(c22 * c33 - c23 * c23 > 0.0))
            return nfail(err, err_len, ALF_ERR_NONPHYSICAL_MATERIAL, "alf_solve_field_noalloc: material");
        MatD d{};
        d.a22 = c22 / rho;
        d.a23 = c23 / rho;
        d.a33 = c33 / rho;
        d.a44 = c44 / rho;
        d.iso = (c22 == c33 && c23 == c22 - 2.0 * c44) ? 1 : 0;
        mats[m] = d;
        for (int k = 0; k < 180; ++k) {
            const double th = k * 3.141592653589793 / 180.0, c = std::cos(th), s = std::sin(th);
            double lam = d.a22;
            if (!d.iso) {
                const double al = c * c * d.a22 + s * s * d.a44, ga = c * c * d.a44 + s * s * d.a33;
                const double be = c * s * (d.a23 + d.a44);
                lam = 0.5 * ((al + ga) + std::sqrt((al - ga) * (al - ga) + 4.0 * be * be));
            }
            vmax = std::max(vmax, std::sqrt(lam));
        }
    }
    if (cudaSetDevice(cuda_device) != cudaSuccess)
        return nfail(err, err_len, ALF_ERR_CUDA, "alf_solve_field_noalloc: cudaSetDevice failed");
    unsigned char* S = nullptr;
    if (scratch_address(&S) != cudaSuccess)
        return nfail(err, err_len, ALF_ERR_CUDA, "alf_solve_field_noalloc: cudaGetSymbolAddress failed");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    FieldDesc fd{};
    fd.node_off = 0;
    fd.map_off = 0;
    fd.nx = nx;
    fd.ny = ny;
    fd.sample = 0;
    fd.si = si;
    fd.sj = sj;
    fd.cell_time = h / vmax;
    QueueState q0{};
    const size_t N = (size_t)nx * ny;
    size_t bm_off = 0;
    unsigned long long pending = 0;
    cudaError_t e = cudaSuccess;
    // inputs of the scratch (small, from the host) and the words that must start at zero
    if (e == cudaSuccess) e = cudaMemcpyAsync(S + kOffQ, &q0, sizeof(q0), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S + kOffField, &fd, sizeof(fd), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S + kOffMats, mats, sizeof(MatD) * nmaterials, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S + kOffH, &h, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S + kOffFrozen, 0, sizeof(unsigned) * kFrozenWords, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S + kOffCounters, 0, 128, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S + kOffCounters + 48, &bm_off, sizeof(size_t), cudaMemcpyHostToDevice, st);
    // every region and material id in range before any kernel indexes with them
    unsigned bad = 0u;
    if (e == cudaSuccess) {
        const int blocks = std::max(1, std::min(device_sm_count() * 4, (int)((N + 255) / 256)));
        check_ids_kernel<<<blocks, 256, 0, st>>>(region_map, (int)N, region_material, nregions, nmaterials,
                                                 (uint32_t*)(S + kOffMap32), (uint32_t*)(S + kOffRmat32),
                                                 (unsigned*)(S + kOffCounters + 96));
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, S + kOffCounters + 96, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && bad != 0u)
        return nfail(err, err_len, ALF_ERR_INVALID_ARG,
                     "alf_solve_field_noalloc: a region id >= nregions or a material id >= nmaterials");
    const FieldDesc* d_fd = (const FieldDesc*)(S + kOffField);
    const uint32_t* d_map32 = (const uint32_t*)(S + kOffMap32);
    const uint32_t* d_rmat32 = (const uint32_t*)(S + kOffRmat32);
    const MatD* d_mats = (const MatD*)(S + kOffMats);
    const double* d_h = (const double*)(S + kOffH);
    unsigned* d_frozen = (unsigned*)(S + kOffFrozen);
    QueueState* d_q = (QueueState*)(S + kOffQ);
    unsigned* ctr = (unsigned*)(S + kOffCounters);
    if (e == cudaSuccess)
        e = launch_prep_regions(ALF_FP32, d_mats, d_rmat32, region_theta, d_h, 1, nregions, group_model,
                                S + kOffRegions, st);
    if (e == cudaSuccess) e = launch_fill_inf(ALF_FP32, times, N, st);
    if (e == cudaSuccess)
        e = launch_init_radius(ALF_FP32, times, d_fd, 1, d_map32, d_rmat32, d_mats, region_theta, d_h,
                               nregions, init_radius, group_model, d_frozen, init_radius, st);
    FimLaunch a{};
    a.times = times;
    a.fields = d_fd;
    a.nfields = 1;
    a.region_map = d_map32;
    a.regions = S + kOffRegions;
    a.nregions = nregions;
    a.box = init_radius;
    a.list[0] = (unsigned*)(S + kOffList0);
    a.list[1] = (unsigned*)(S + kOffList1);
    a.elist = (unsigned*)(S + kOffElist);
    a.bitmap = (unsigned*)(S + kOffBitmap);
    a.cnt = ctr;             // [2]
    a.ecnt = ctr + 2;        // [1]
    a.eoff = ctr + 4;        // [2]
    a.rounds = ctr + 6;      // [1]
    a.bm_off = (const size_t*)(S + kOffCounters + 48);
    a.flim = S + kOffCounters + 64;
    a.efield = (unsigned*)(S + kOffEfield);
    a.oldv = S + kOffOld;
    a.newv = S + kOffNew;
    // the host counts the rounds against the cap (64 (nx + ny) unless given); the device's own cap lies
    // beyond it.  The front band is the plan's default, 2 cell-crossing times.
    const long long max_total = max_rounds > 0 ? (long long)max_rounds : 64ll * (nx + ny);
    a.max_rounds_per_node = (unsigned)(max_total / (nx + ny) + 2);
    a.band_cells = 2.0;
    a.q = d_q;
    a.records = nullptr;
    unsigned long long* d_pending = (unsigned long long*)(S + kOffCounters + 56);
    if (e == cudaSuccess) e = launch_fim_init(ALF_FP32, a, 1, st);
    int parity = 0;
    const int grid_eval = device_sm_count() * 16;
    for (long long r = 0; e == cudaSuccess && r < max_total;) {
        for (int k = 0; k < 32 && r < max_total && e == cudaSuccess; ++k, ++r) {
            e = launch_fim_round(ALF_FP32, a, parity, 1, grid_eval, st);
            parity ^= 1;
        }
        if (e == cudaSuccess) e = launch_fim_pending(a, parity, d_pending, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&pending, d_pending, sizeof(pending), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && pending == 0ull) break;
    }
    if (e == cudaSuccess)
        e = launch_finalize(ALF_FP32, times, d_fd, 1, init_radius, nullptr, 1, 0, nullptr, nullptr, st);
    QueueState qh{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&qh, d_q, sizeof(qh), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        std::snprintf(msg, sizeof(msg), "alf_solve_field_noalloc: %s", cudaGetErrorString(e));
        return nfail(err, err_len, ALF_ERR_CUDA, msg);
    }
    if (qh.error != 0u || pending != 0ull)
        return nfail(err, err_len, ALF_ERR_NOT_CONVERGED,
                     "alf_solve_field_noalloc: the sweep reached its round cap before the fixed point");
    return nfail(err, err_len, ALF_OK, "");
}
