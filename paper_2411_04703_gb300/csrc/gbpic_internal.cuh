// Internal declarations of the gbpic CUDA library (sm_103a).  Device-side parameter blocks,
// the context structure and the kernel launchers used by the C-ABI in api.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "gbpic.h"

namespace gbpic {

constexpr int kMaxSpecies = 8;
constexpr int kChunk = 4096;         // particles per work item of the particle kernel (at most)
constexpr int kChunkMin = 512;       // smallest work item (small species are split finer)
constexpr int kPushThreads = 1024;   // 32 warps per SM at 64 registers (measured 3 % faster than 512 at 122)
constexpr int kGroup = kChunk / kPushThreads;   // consecutive particles of one lane per work item
constexpr int kSparse = 32;   // a tile with fewer particles takes the global-memory path, one warp per tile

// Error bits of the device error word.
enum : int {
    ERR_INDEX = 1,      // a slow-path stencil node fell outside a non-periodic grid
    ERR_CAPACITY = 2,   // an append (load / injection) exceeded the species capacity
    ERR_MOVE = 4,       // a particle moved one cell or more in one step (Courant violated)
    ERR_NAN = 8,        // non-finite momentum produced by the push
};

// Cell index packed into 31 bits: i | j << sj | k << sk, with sj the bits of nx and sk - sj
// the bits of ny (set per context); -1 marks a dummy particle.
struct CellCode {
    int sj, sk, mi, mj;
    __host__ __device__ __forceinline__ int pack(int i, int j, int k) const { return i | (j << sj) | (k << sk); }
    __host__ __device__ __forceinline__ int i(int c) const { return c & mi; }
    __host__ __device__ __forceinline__ int j(int c) const { return (c >> sj) & mj; }
    __host__ __device__ __forceinline__ int k(int c) const { return c >> sk; }
};

// Ensembles: `runs` independent runs of nzr cells along z are stacked along z in one grid; z is
// periodic inside each run's block of rows [b, b + nzr), b a multiple of nzr.  A single run has
// nzr = nz.
__host__ __device__ __forceinline__ int zblock(int k, int nzr) { return (k / nzr) * nzr; }
__host__ __device__ __forceinline__ int zwrap(int k, int b, int nzr) { return k < b ? k + nzr : (k >= b + nzr ? k - nzr : k); }

// Index p of a periodic dim of n cells brought into [0, n): one step for the usual offsets of a
// stencil, a remainder when the dim is shorter than the stencil (n = 1: a 2-D geometry).
__host__ __device__ __forceinline__ int pwrap(int p, int n)
{
    if (p < 0) p += n;
    else if (p >= n) p -= n;
    if (p < 0 || p >= n) p = ((p % n) + n) % n;
    return p;
}

struct GridDev {
    int n[3];
    int periodic[3];
    float d[3];
    float dt;
    float dt_over_d[3];
    int mlo, mhi;        // particle margins of the non-periodic dims
    long long ncell;
    CellCode cc;
    int nzr;             // rows per run along z (z wraps inside a run's block when periodic)
};

struct PmlDev {
    int on;
    const float *bE[3];   // exp(-sigma(node) dt) per dim, size n[d]
    const float *bB[3];   // exp(-sigma(node + 1/2) dt/2) per dim, size n[d]
    float *psiE;          // [6][ncell]: (Ex,y) (Ex,z) (Ey,z) (Ey,x) (Ez,x) (Ez,y)
    float *psiB;          // [6][ncell]: same order for B
};

struct ExtDev {
    int type;             // PIC_EXT_*
    float B0g;            // gamma_R B0 (RRF amplitude of B'_y)
    float beta_R;
    float kdz;            // k'_u dz: phase advance per cell along z
    float theta;          // phase of the step: k'_u (shifts dz + beta_R t') + phase, mod 2 pi
    const float *phase_tab;  // (k'_u dz k) mod 2 pi for k = 0 .. nz-1
    int ramp_mode;        // 0: f = 1; 1: linear ramp; 2: step
    float ramp_a, ramp_b; // ramp argument r = ramp_a (k + off_z) + ramp_b
    const float *amp_tab; // ensembles: gamma_R B0 of the run that owns row k; NULL: B0g everywhere
    float kuy;            // 3-D field: k_u dy, the phase of cosh / sinh per cell along y
    float y0;             // 3-D field: undulator axis (grid y coordinate of the mid-plane)
    float igR;            // 1 / gamma_R (B'_z = B_z = B'_y amplitude / gamma_R)
    // the step's phase and ramp offset from the device step counter (so that a captured CUDA
    // graph replays correctly): theta = (th_a n + th_b) mod 2 pi, ramp_b = rb_a n + rb_b
    const long long *clock;
    double th_a, th_b, rb_a, rb_b;
};

// The external field of the current step, from the device step counter.
__device__ __forceinline__ ExtDev ext_at_clock(const ExtDev &e)
{
    ExtDev x = e;
    if (e.type && e.clock) {
        const double n = (double)*e.clock;
        x.theta = (float)fmod(e.th_a * n + e.th_b, 6.283185307179586);
        x.ramp_b = (float)(e.rb_a * n + e.rb_b);
    }
    return x;
}

struct SpeciesDev {
    float4 *pos;          // (off_x, off_y, off_z, cell bits)
    float4 *mom;          // (u_x, u_y, u_z, w)
    int *id;
    int *count;           // [0] total slots in use, [1] sorted prefix, [2] tile work items
    float h_qm;           // 0.5 (q/m) dt
    float cf[3];          // -q d_c / (dt V): current of unit weight per unit W
    // Fixed-point scale of the shared-memory current, set per work item: a contribution is at most
    // jb_c w |d_c| (w the largest weight, d_c the displacement), and the scale maps the bound
    // jb_c w dlim_c to at most 2^30.  dlim is adaptive: four times the largest |d_c| of the
    // previous step; a particle moving further deposits with float atomics.
    float jb[3];          // 1.1 |cf_c|
    float wmax;           // largest |weight| the species holds
    const float *wrun;    // ensembles: largest |weight| of each run; NULL: wmax everywhere
    const float *dlim;    // device [3]: displacement bound of this step (cells)
    unsigned *dmax;       // device [3]: largest |displacement| of this step (float bits, atomicMax)
    unsigned long long *nfall;  // device counter of particles that took the float-atomic fallback
    int pusher;           // PIC_PUSHER_BORIS or PIC_PUSHER_VAY
    int frozen;
    int cap;
};

struct TileDev {
    int T[3];             // tile size (cells)
    int nt[3];            // tiles per dim
    int tile_cells;
    int M;                // allowed drift outside the tile between sorts (cells)
    int hl;               // stencil reach below the particle cell (1 CIC, 2 TSC)
    int R[3];             // shared-memory region size per dim
    const int *cell_start;   // [n_keys + 1]: first sorted slot of each key (8 keys per cell), valid
                             // for the tiles holding particles at the last sort
    const int *tile_start;   // [ntiles + 1]: first sorted slot of each tile (the last: the live count)
    const int2 *items;       // (tile, chunk) work items of the tiles with >= kSparse particles
    const int *sparse_tiles; // tiles with 1 .. kSparse-1 particles (count[3] of them)
    int chunk;               // particles per work item (kChunkMin .. kChunk), fixed at the sort
    CellCode cc;
};

struct FieldsDev {
    float *E, *B, *J;     // [3][ncell] each
};

// One plane of the lab-static plasma lattice, held by a lattice species (the frozen plasma
// ions): every ion of plane m shares the z offset, the cell row and the weight, and ion r of
// the plane (r over the transverse lattice, as injected) has id id0 + r.
struct PlaneRec {
    float oz;             // z offset in the cell
    int kz;               // cell row; -1: the plane was dropped (or never placed)
    float w;              // macroparticle weight
    int id0;
};

// Particle shape of order 1 (CIC) or 2 (TSC) at distance x from a node, FP64 (the lattice
// species' current and transverse profiles; the particle kernel uses its own FP32 forms).
__device__ __forceinline__ double shape_weight(int order, double x)
{
    const double a = fabs(x);
    if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
    if (a <= 0.5) return 0.75 - a * a;
    if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
    return 0.0;
}

// ------------------------------------------------------------------------- host context
struct Species {
    double q = -1, m = 1;
    int frozen = 0;
    int64_t cap = 0;
    float4 *pos = nullptr, *mom = nullptr, *pos2 = nullptr, *mom2 = nullptr;
    int *id = nullptr, *id2 = nullptr;
    int *count = nullptr;     // device [4]
    int *rank = nullptr;      // device [cap] sort scratch
    int2 *items = nullptr;    // device work items
    int64_t max_items = 0;
    int *cell_start = nullptr;  // device [n_keys + 1]; zero outside the tiles listed in occ
    int *tile_start = nullptr;  // device [ntiles + 1]: particles per tile, then their exclusive scan
    int *occ = nullptr;         // device [ntiles + 1]: the tiles holding particles at the last sort;
                                // occ[ntiles] counts them
    int *chunk_start = nullptr; // device [ntiles + 1]
    int *sparse_start = nullptr;  // device [ntiles + 1]: scan of the sparse-tile flags
    int *sparse_tiles = nullptr;  // device [ntiles]: the sparse tiles
    int chunk = kChunk;           // particles per work item, chosen at each sort
    int64_t bound = 0;        // host upper bound of count[0]
    int64_t next_id = 0;
    double wmax = 0;          // largest |weight| ever held (sets the fixed-point current scale)
    std::vector<double> wmax_run;  // ensembles: largest |weight| ever held in each run
    float *wrun = nullptr;    // device [runs] copy of wmax_run (ensembles)
    float *dlim = nullptr;    // device [3] adaptive displacement bound of the current deposit
    unsigned *dmax = nullptr; // device [3] largest displacement measured in the last push
    // lattice species (plasma ions): no particle records, a ring of lattice planes instead
    int lattice = 0;
    PlaneRec *planes = nullptr;  // device [plane_cap]; plane m in slot m mod plane_cap
    int64_t plane_cap = 0;
    float *tx = nullptr, *ty = nullptr;   // device [n0], [n1]: node weights summed over the transverse lattice
    double *zacc = nullptr;      // device [n2]: J_z per unit transverse weight, one step
};

// Saved state of the run (a checkpoint of the adjoint, or one recorded step of a segment).
struct SpeciesSnap {
    float4 *pos = nullptr, *mom = nullptr;
    int *id = nullptr;
    int *dcount = nullptr;     // device copy of the species' count[4] (recorded steps)
    int n = 0;                 // slots in use
    int count[4] = {0, 0, 0, 0};
    float dlim[4] = {0, 0, 0, 0};
    PlaneRec *planes = nullptr;   // lattice species
};
struct StateSnap {
    int64_t step = 0;
    bool sorted = false;       // recorded step: the step began with a sort
    float *E = nullptr, *B = nullptr;
    std::vector<SpeciesSnap> sp;
};

}  // namespace gbpic

struct pic_ctx {
    pic_device dev{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int n[3] = {0, 0, 0};
    int runs = 1, nzr = 0;        // ensemble: runs stacked along z, nzr rows each
    gbpic::CellCode cc{};
    double d[3] = {0, 0, 0};
    double dt = 0, gR = 1, bR = 0;
    int bc[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    int pml = 0;
    int moving = 0;
    double vw = 0;
    int order = 1;
    int64_t ncell = 0;
    float *E = nullptr, *B = nullptr, *J = nullptr, *rho = nullptr;
    float *psiE = nullptr, *psiB = nullptr;
    float *pml_coef = nullptr;   // bE[3][nmax], bB[3][nmax]
    float **shift_tab = nullptr; // device table of the arrays the moving window shifts
    int shift_n = 0;
    int nmax = 0;
    // external field
    int ext_type = 0;
    double K = 0, lam_u = 0, ku = 0, B0 = 0, phase0 = 0, z_start = 0, ramp = -1;
    float *phase_tab = nullptr;
    std::vector<double> B0_run;   // ensembles: B0 of each run (empty: B0 for every run)
    float *amp_tab = nullptr;     // ensembles: device [nz] gamma_R B0 of the run owning row k
    std::vector<double> dens_run; // ensembles: plasma density scale of each run
    // plasma
    int plasma = 0, sp_e = -1, sp_i = -1, ppc[3] = {1, 1, 1}, xr[4] = {0, 0, 0, 0};
    double *prof = nullptr;   // device [2][nprof]
    double *dens_scale = nullptr;  // ensembles: device [runs] density scale of each run
    int nprof = 0;
    std::vector<double> prof_z, prof_n;
    // tiles
    int T[3] = {8, 8, 8};
    int sort_every = 8;
    int64_t sort_base = 0;        // pic_step sorts when (step - sort_base) % sort_every == 0
    int M = 1;
    int nt[3] = {1, 1, 1};
    int ntiles = 1;
    int64_t n_keys = 1;
    int *hist_tmp = nullptr;      // scan scratch
    int64_t hist_tmp_n = 0;
    // time
    int64_t step = 0, shifts = 0, m_last = -1;
    // bookkeeping
    int *err = nullptr;           // device error word
    long long *dclock = nullptr;  // device step counter (equals step; advanced by a kernel per step)
    // CUDA graph of whole sort periods (no moving window, no injection, tracing off)
    int use_graphs = 1;
    int pusher = 0;               // PIC_PUSHER_*
    int gather = 0;               // PIC_GATHER_*
    // artificial neutralising ions fading over [ion_t0, ion_t0 + ion_T]: their J_z is ion_G / ion_T
    float *ion_G = nullptr;
    double ion_t0 = 0, ion_T = 0;
    // lab-frame snapshot of species snap_sp at lab time snap_T (time-skew reconstruction): by
    // particle id, lab x, y, z, u_x, u_y, u_z, w (FP64) and a state (0 pending, 1 recorded, 2 missed)
    double *snap = nullptr;
    unsigned char *snap_state = nullptr;
    int snap_sp = -1;
    int64_t snap_n = 0;
    double snap_T = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_steps = 0;      // steps one replay advances
    int64_t graph_kernels = 0;    // kernels one replay runs
    const void *graph_key = nullptr;   // first species' particle array when captured (pointer parity)
    // adjoint: checkpoints every ad_every steps from ad_step0; while a segment is recomputed,
    // every step's post-sort state is recorded into ad_rec[ad_rec_n++]
    int ad_on = 0, ad_every = 0;
    int64_t ad_step0 = 0;
    std::vector<gbpic::StateSnap> ad_ckpt;
    std::vector<gbpic::StateSnap> ad_rec;
    int ad_rec_n = -1;         // < 0: not recording
    unsigned long long *nfall = nullptr;   // device counter of fallback deposits (tracing)
    int *work = nullptr;          // device work counters [2 * kMaxSpecies]
    double *red = nullptr;        // reduction partials
    double *red_out = nullptr;
    int nsp = 0;
    gbpic::Species sp[gbpic::kMaxSpecies];
    std::string msg;
    bool poisoned = false;
    std::vector<std::pair<void *, size_t>> allocs;   // every device allocation of the context
    // tracing
    bool trace_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    double trace_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t trace_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t kernels = 0;          // kernels launched since the last trace read
};

namespace gbpic {

GridDev grid_dev(const pic_ctx *c);
TileDev tile_dev(const pic_ctx *c, const Species &s);
SpeciesDev species_dev(const pic_ctx *c, const Species &s);
ExtDev ext_dev(const pic_ctx *c);
PmlDev pml_dev(const pic_ctx *c);

// k_push.cu
cudaError_t launch_push(pic_ctx *c, int si, const ExtDev &ext);
cudaError_t launch_dlim_from_momenta(pic_ctx *c, int si);
cudaError_t launch_rho(pic_ctx *c, const Species &s, float *rho);
// k_lattice.cu
cudaError_t launch_lattice_profiles(pic_ctx *c, int si);
cudaError_t launch_lattice_step(pic_ctx *c, int si);
cudaError_t launch_lattice_shift(pic_ctx *c, int si);
cudaError_t launch_lattice_records(pic_ctx *c, int si, Species &out);
// k_fields.cu
cudaError_t launch_fdtd_b(pic_ctx *c, float dtt);
cudaError_t launch_fdtd_e(pic_ctx *c);
cudaError_t launch_shift_fields(pic_ctx *c);
cudaError_t launch_field_energy(pic_ctx *c, double *out_host, int run);
cudaError_t launch_ion_prefix(pic_ctx *c, const float *rho, float *G);
cudaError_t launch_ion_current(pic_ctx *c, float f);
cudaError_t launch_ion_shift(pic_ctx *c);
// k_snapshot.cu
cudaError_t launch_snap_arm(pic_ctx *c);
cudaError_t launch_snap_record(pic_ctx *c);
cudaError_t launch_snap_moments(pic_ctx *c, double k, double *out);
// k_sort.cu
cudaError_t launch_sort(pic_ctx *c, int si);
cudaError_t exclusive_scan(pic_ctx *c, int *data, int64_t n);
int64_t scan_scratch_size(int64_t n);
// k_init.cu
cudaError_t launch_load(pic_ctx *c, int si, int64_t n, const double *dx, const double *du,
                        const double *dw, int frame, const double origin[3], int match,
                        int64_t id_base, int run, int64_t stride);
cudaError_t launch_inject(pic_ctx *c, int64_t m0, int64_t m1);
cudaError_t launch_shift_particles(pic_ctx *c, int si);
cudaError_t launch_moments(pic_ctx *c, const Species &s, int frame, double k, double *out20, int run);
cudaError_t species_wmax(pic_ctx *c, int si, double *out);
cudaError_t species_count_live(pic_ctx *c, const Species &s, int64_t *out);
cudaError_t absmax_f64(pic_ctx *c, const double *a, int64_t n, double *out);
// k_adjoint.cu
cudaError_t adj_fields(pic_ctx *c, float *lE, float *lB, float *lJ);
cudaError_t adj_particles(pic_ctx *c, const Species &rec, const float *E, const float *B, const float *lJ, float *lE,
                          float *lB, float4 *lx, float4 *lu, double *lw, double *lK, const ExtDev &ext, int n);
cudaError_t adj_ions(pic_ctx *c, const Species &s, const PlaneRec *planes, const float *lJ, double *R, double *lw_plane);
cudaError_t adj_bunch_seed(pic_ctx *c, const Species &s, double k, double *sums_dev, double *host3, float4 *lx);
cudaError_t adj_remap(pic_ctx *c, const int *id_before, int n_before, const int *id_after, int n_after, int *inv,
                      const float4 *lx, const float4 *lu, float4 *lx_out, float4 *lu_out);
cudaError_t adj_profile_grad(pic_ctx *c, const double *lw_e, long long n_ids, const double *lw_plane, double *grad);

}  // namespace gbpic
