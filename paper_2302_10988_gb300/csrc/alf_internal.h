// alf_internal.h -- types shared by the library's translation units (host side).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/alifmm.h"
#include "alf_device.cuh"

namespace alf {

// One field (sample b, source s) in the packed layout.
struct FieldDesc {
    long long node_off;  // first node in the packed times buffer
    long long map_off;   // first node of the sample's region map
    int nx, ny;
    int sample;
    int si, sj;          // source node
    int pad;
    double cell_time;    // h / (fastest group speed of the materials): time to cross one cell
};

// Device-side counters and status words of one solve.
struct QueueState {
    unsigned head;              // next field to take
    unsigned error;             // alf_status of the first device failure
    unsigned long long visits;  // node evaluations queued over all rounds
    unsigned long long rounds;  // rounds over all fields
    unsigned long long dirty;   // dirty-list entries scanned over all rounds (field-resident schedules)
};

struct FimLaunch {
    void* times;
    const FieldDesc* fields;
    int nfields;
    const uint32_t* region_map;
    const void* regions;  // RegionP<T>[nsamples][nregions]
    int nregions;
    int box;                       // half-width of the frozen box around each source
    unsigned* list[2];             // dirty lists, segments at the fields' node offsets
    unsigned* elist;               // evaluation lists, same segments
    unsigned* bitmap;              // dirty bitmaps, field f at word bm_off[f]
    const size_t* bm_off;
    unsigned* cnt;                 // [2][nfields] dirty-list sizes (by round parity)
    unsigned* ecnt;                // [nfields] evaluation-list sizes
    unsigned* eoff;                // [nfields + 1] exclusive scan of ecnt
    unsigned* efield;              // [total nodes] field of each evaluation slot
    void* oldv;                    // [total nodes] time before / after each evaluation
    void* newv;
    unsigned* rounds;              // [nfields] rounds taken
    void* flim;                    // [nfields] T + band of the current round
    unsigned max_rounds_per_node;  // round cap = this x (nx + ny)
    double band_cells;             // evaluation band beyond the front, in cells of cell_time (<= 0: none)
    QueueState* q;
    uint8_t* records;
    int vtable;                    // the regions carry velocity tables (kernels compiled with the lookup)
    // FP64 check fused into the CTA sweep (launch_fim_cta with check): RegionP<double>, frozen bitmaps, outputs
    const void* regions64 = nullptr;
    const unsigned* frozen_bits = nullptr;
    double* max_rel = nullptr;
    int32_t* n_flips = nullptr;
};

// kernels (alf_kernels.cu)
// velocity table: the qP phase speed at 0, 1, ..., 180 degrees from the material axis, per material
#define ALF_VTAB_N 181
cudaError_t launch_prep_regions(int precision, const MatD* mats, const uint32_t* region_mat, const double* theta,
                                const double* h, int nsamples, int nregions, int group_model, void* regions_out,
                                cudaStream_t st, const void* vtab = nullptr);
cudaError_t launch_fill_inf(int precision, void* times, size_t n, cudaStream_t st);
// the shear modes' group slownesses: ALF_ENV_N entries per material (mats[].env ignored)
cudaError_t launch_env_table(const MatD* mats, int nmat, double* tab, cudaStream_t st);
// records `code` in q->error unless an earlier failure is recorded there (one tiny launch)
cudaError_t launch_set_status(QueueState* q, unsigned code, cudaStream_t st);
// streaming multiprocessors of the current device (queried once per device)
int device_sm_count();
cudaError_t launch_init_radius(int precision, void* times, const FieldDesc* fields, int nfields,
                               const uint32_t* region_map, const uint32_t* region_mat, const MatD* mats,
                               const double* theta, const double* h, int nregions, int r0, int group_model,
                               unsigned* frozen_bits, int box, cudaStream_t st);
cudaError_t launch_fim_init(int precision, const FimLaunch& a, int grid_fields, cudaStream_t st);
cudaError_t launch_fim_round(int precision, const FimLaunch& a, int parity, int grid_fields, int grid_eval,
                             cudaStream_t st, int eval_block = 128, cudaEvent_t ev0 = nullptr,
                             cudaEvent_t ev1 = nullptr);
// kernel launches issued by this library so far (all plans, all devices)
void note_launches(unsigned n);
unsigned long long launches_so_far();
cudaError_t launch_fim_pending(const FimLaunch& a, int parity, unsigned long long* out, cudaStream_t st);
// field-resident sweep: one warp per field, fields taken in the order `order`
#define ALF_SWEEP_WARPS 4
cudaError_t launch_fim_warp(int precision, const FimLaunch& a, const unsigned* order, unsigned words_per_warp,
                            int grid, cudaStream_t st);
int fim_warp_ctas_per_sm(int precision, unsigned words_per_warp, bool vt);  // 0: does not fit
// field-resident sweep by a CTA per field (few large fields); bitmaps of up to smem_words words in shared memory
// (threads: 64..512 per CTA; cluster: 1, or 2 / 4 / 8 CTAs of 512 threads sharing one field)
cudaError_t launch_fim_cta(int precision, const FimLaunch& a, const unsigned* order, unsigned smem_words, int grid,
                           int threads, int cluster, cudaStream_t st, bool check = false);
// the CTA sweep can run each field's FP64 check itself (FP32, no velocity table, one CTA per field)
bool fim_cta_can_check(int precision, int vtable, int cluster);
int fim_cta_grid(int precision, unsigned smem_words, bool vt, int threads, int cluster, int nsm);  // CTAs; 0: none
// active-tile sweep (alf_tile.cu): one CTA of 8 warps per field, 8 x 8 tiles iterated in shared memory; the
// tile bitmap of a field in shared memory when it has at most smem_words words (fim_tile_words), else global
cudaError_t launch_fim_tile(int precision, const FimLaunch& a, const unsigned* order, unsigned smem_words, int grid,
                            cudaStream_t st);
int fim_tile_grid(int precision, unsigned smem_words, bool vt, int nsm);  // CTAs resident at once; 0: none
unsigned fim_tile_words(int nx, int ny);                                  // words of a field's tile bitmap
cudaError_t launch_finalize(int precision, void* times, const FieldDesc* fields, int nfields, int box,
                            const int32_t* rec_ij, int nsrc, int nrec, void* rec_times, uint8_t* records,
                            cudaStream_t st);
cudaError_t launch_check64(int precision, const void* times, const FieldDesc* fields, int nfields,
                           const uint32_t* region_map, const void* regions64, int nregions, const uint8_t* records,
                           const unsigned* frozen_bits, int box, double* max_rel, int32_t* n_flips, int grid_ctas,
                           cudaStream_t st, int vtable = 0, double* F_out = nullptr, uint8_t* rec_out = nullptr);
cudaError_t launch_eval_velocity(const MatD* mat, int kind, int group_model, int precision, const double* angles,
                                 double* out, int n, cudaStream_t st);

// near-source hierarchy (alf_hier.cu)
struct HierLaunch {
    void* times;
    const FieldDesc* fields;
    int nfields;
    const uint32_t* region_map;
    const uint32_t* region_mat;
    const MatD* mats;
    const void* regions;  // RegionP<T>
    const double* theta;
    const double* h;
    int nregions;
    int group_model;
    int nlev;
    int dens[4];
    int rad[4];
    int box;                 // = rad[nlev - 1]: half-width of the frozen box on the original grid
    unsigned* frozen_bits;
    size_t level_cap;        // nodes of the largest level grid
    void* scratch;           // per warp: scratch_stride bytes
    size_t scratch_stride;   // hier_scratch_bytes(precision, level_cap)
    int nwarps;              // warps launched (one field at a time each)
    unsigned* head;          // field counter
    QueueState* q;           // error word
    double band_cells;
    unsigned max_rounds_per_node;
    int vtable;
};
size_t hier_scratch_bytes(int precision, size_t level_cap);
cudaError_t launch_init_hierarchy(int precision, const HierLaunch& a, cudaStream_t st);

// adjoint (alf_adjoint.cu)
struct AdjLaunch {
    const void* times;
    const FieldDesc* fields;
    int nfields, nsamples, nrec;
    size_t total_nodes;
    const uint32_t* region_map;
    const uint32_t* region_mat;
    const MatD* mats;
    const void* regions;  // RegionP<T>
    const double* theta;
    const double* h;
    int nregions;
    int box;
    int group_model;
    const unsigned* frozen_bits;
    const uint8_t* records;
    const int32_t* rec_ij;
    void* nodes;      // per node: AdjNode<T> (weights, lambda, lambda * dtau/dtheta, in-degree)
    unsigned* list[2];
    unsigned* cnt;    // [2][nfields]
    unsigned* eoff;   // [nfields + 1]
    unsigned max_rounds;
    // field-resident schedule (one warp per field, one launch): fields by decreasing size, a work
    // counter, and the number of warps to launch (0: lockstep rounds over all fields instead)
    const unsigned* order;
    unsigned* head;
    int warp_grid;
    QueueState* q;    // status word: a node never released by the Kahn sweep records ALF_ERR_INCONSISTENT_RECORDS
};
size_t adj_node_bytes(int precision);
cudaError_t launch_adjoint(int precision, const AdjLaunch& a, const void* dL_drec, double* grad,
                           unsigned long long* d_pending, unsigned long long* h_pending, int grid, cudaStream_t st);

// rays (alf_ray.cu)
struct RayLaunch {
    const void* times;
    const FieldDesc* fields;
    int nfields;
    const uint32_t* region_map;
    const uint32_t* region_mat;
    const MatD* mats;
    const void* regions;  // RegionP<T>
    const double* theta;
    int nregions;
    const int32_t* rec_ij;
    int nsrc, nrec;
    int group_model;
    int plane_step, halfwidth, max_pts;
    int family;  // -1: the plane set most perpendicular at every step; 0..3: one fixed set; 4: fastest of the four
    const double* h_of_sample;  // grid spacing of every sample (device)
    double stop_radius;
    void* pts;
    int32_t* npts;
    void* ray_time;
    int32_t* ray_status;
    unsigned* error;
};
cudaError_t launch_rays(int precision, const RayLaunch& a, cudaStream_t st);
// packed ray points: offsets[nrays + 1] (int64) and the points back to back; block_sums: (nrays + 1023) / 1024 + 1
cudaError_t launch_pack_rays(int precision, const void* pts, const int32_t* npts, long long nrays, int max_pts,
                             long long* block_sums, void* packed, long long* offsets, int grid, cudaStream_t st);
// gradient of the ray times along the given paths (a.pts, a.npts) by the region orientations
cudaError_t launch_ray_gradient(int precision, const RayLaunch& a, const void* dL_dray, double* grad, int nsamples,
                                cudaStream_t st);

}  // namespace alf

struct alf_ctx {
    int device = 0;
    int nsm = 0;
    int cc_major = 0, cc_minor = 0;
    std::string err;
    alf::MatD* d_scratch_mat = nullptr;
    double* d_scratch_env = nullptr;  // one material's envelope table (alf_eval_velocity)
};

struct alf_plan {
    alf_ctx* ctx = nullptr;
    alf_options opt{};         // in effect: lengths in cells of the (sub-grid refined) plan grid
    alf_options opt_caller{};  // as given, lengths in original cells
    int B = 0, S = 0, Rr = 0, R = 0, nmat = 0, nfields = 0;
    std::vector<alf::FieldDesc> fields;
    std::vector<size_t> field_off;
    size_t total_nodes = 0;
    size_t total_map = 0;
    size_t max_field_nodes = 0;
    int grid_fields = 0;  // CTAs of the per-field sweep steps (one warp per field)
    int grid_eval = 0;    // CTAs of the flat evaluation and marking steps
    size_t bm_words = 0;
    int box = 0;  // half-width of the frozen box around each source
    // device
    alf::FieldDesc* d_fields = nullptr;
    uint32_t* d_map = nullptr;  // region id of every node, samples back to back
    uint32_t* d_region_mat = nullptr;
    alf::MatD* d_mats = nullptr;
    double* d_h = nullptr;
    int32_t* d_rec = nullptr;
    void* d_regions = nullptr;    // RegionP<T> of the plan precision
    void* d_regions64 = nullptr;  // RegionP<double> for the FP64 check
    void* d_vtab = nullptr;          // velocity tables of the plan precision (option velocity_table)
    double* d_vtab64 = nullptr;      // the same in FP64, for the FP64 check
    void* d_regions_rays = nullptr;  // RegionP<T> of the ray tracer (its own copy: rays may overlap the others)
    double* d_env = nullptr;         // shear modes: ALF_ENV_N envelope slownesses per material
    // sweep workspace
    unsigned* d_list0 = nullptr;
    unsigned* d_list1 = nullptr;
    unsigned* d_elist = nullptr;
    unsigned* d_efield = nullptr;
    void* d_oldv = nullptr;
    void* d_newv = nullptr;
    unsigned* d_bitmap = nullptr;
    size_t* d_bm_off = nullptr;
    unsigned* d_cnt = nullptr;
    unsigned* d_ecnt = nullptr;
    unsigned* d_eoff = nullptr;
    unsigned* d_rounds = nullptr;
    void* d_flim = nullptr;
    unsigned long long* d_pending = nullptr;
    unsigned long long* h_pending = nullptr;  // pinned
    int rounds_per_check = 32;
    // field-resident sweep (option sweep = 2, or chosen by sweep = 0)
    int sweep_mode = 1;             // 1: bulk-synchronous rounds, 2: one warp per field, 3: one CTA per field,
                                    // 4: active tiles, one CTA per field
    unsigned cta_words = 0;         // shared bitmap words of the CTA-per-field sweep
    int cta_grid = 0;
    unsigned tile_words = 0;        // shared tile-bitmap words of the active-tile sweep (0: global bitmaps)
    int tile_grid = 0;              // its CTAs resident at once (0: it cannot run)
    int cta_threads = 256;          // threads of one field's CTA: 64, 128, 256 or 512
    int cta_default = 256;          // the plan's choice when the options leave it open
    int cta_cluster = 1;            // CTAs (of 512 threads) sharing one field: 1, 2, 4 or 8
    int cluster_default = 1;
    unsigned warp_words = 0;        // dirty-bitmap words of the largest field
    int warp_grid = 0;              // CTAs of the field-resident sweep (0: not possible)
    unsigned* d_order = nullptr;    // fields by decreasing size
    unsigned* d_adj_head = nullptr; // work counter of the field-resident adjoint
    // near-source hierarchy (init_mode = ALF_INIT_HIERARCHY)
    size_t hier_cap = 0;            // nodes of the largest level grid
    int hier_warps = 0;
    void* d_hier = nullptr;         // per-warp level scratch
    unsigned* d_hier_head = nullptr;
    int eval_block = 128;           // threads per CTA of the evaluation step (autotuned)
    // CUDA graph of one chunk of rounds, for the pointers it was captured with
    cudaGraphExec_t chunk_graph = nullptr;
    const void* graph_times = nullptr;
    const void* graph_records = nullptr;
    const void* graph_regions = nullptr;
    // evaluation-kernel timing (alf_plan_stats)
    std::vector<cudaEvent_t> ev;
    double eval_ms = 0.0;
    unsigned long long eval_launches = 0, sweep_rounds = 0;
    // adjoint workspace (keep_records = 1)
    void* d_adj_nodes = nullptr;    // AdjNode<T> per node (32 B FP32, 64 B FP64)
    alf::QueueState* d_q = nullptr;
    unsigned* d_ray_error = nullptr;
    long long* d_ray_blocks = nullptr;  // block sums of alf_pack_rays' scan ((nrays + 1023) / 1024 + 1)
    unsigned* d_frozen = nullptr;  // per-field bitmap of frozen nodes in the source box
    alf::QueueState* h_q = nullptr;  // pinned
};
