// C-ABI of the gbpic library: context, device memory, step orchestration and getters.
// Declared and documented in include/gbpic.h.
#include "gbpic_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>

using namespace gbpic;

namespace {

thread_local std::string g_create_err;

int fail(pic_ctx *c, int code, const std::string &m)
{
    if (c) {
        c->msg = m;
        if (code == PIC_ERR_CUDA || code == PIC_ERR_DEVICE) c->poisoned = true;
    } else {
        g_create_err = m;
    }
    return code;
}

int fail_cuda(pic_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, PIC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return fail_cuda(c, e_, #call);   \
    } while (0)

void *dalloc(pic_ctx *c, size_t bytes)
{
    bytes = std::max<size_t>(bytes, 256);
    void *p = nullptr;
    if (c->dev.alloc) {
        p = c->dev.alloc(bytes, c->dev.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs.emplace_back(p, bytes);
    return p;
}

void dfree(pic_ctx *c, void *p)
{
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); i++) {
        if (c->allocs[i].first != p) continue;
        if (c->dev.free) c->dev.free(p, c->allocs[i].second, c->dev.user);
        else cudaFree(p);
        c->allocs.erase(c->allocs.begin() + i);
        return;
    }
}

template <class T>
int alloc_zero(pic_ctx *c, T **out, size_t count)
{
    *out = static_cast<T *>(dalloc(c, count * sizeof(T)));
    if (!*out) return fail(c, PIC_ERR_ALLOC, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
    CK(cudaMemsetAsync(*out, 0, std::max<size_t>(count * sizeof(T), 1), c->stream));
    return PIC_OK;
}

int margin_lo(const pic_ctx *c) { return c->order == 1 ? 1 : 2; }
int margin_hi(const pic_ctx *c) { return c->order == 1 ? 2 : 3; }

// Largest plasma lattice plane whose grid coordinate at step n (after `shifts` window shifts)
// is below nz - margin_hi: plane m sits at ((m + 1/2)/ppc_z) dz - beta_R t' in the RRF.
int64_t plane_max(const pic_ctx *c, int64_t n, int64_t shifts)
{
    const double thr = (double)(c->n[2] - margin_hi(c));
    const double xv = (double)c->ppc[2] * (thr + (double)shifts + c->bR * (double)n * c->dt / c->d[2]) - 0.5;
    return (int64_t)std::ceil(xv) - 1;
}

int check_ctx(pic_ctx *c)
{
    if (!c) return PIC_ERR_ARG;
    if (c->poisoned) return PIC_ERR_STATE;
    return PIC_OK;
}

void drop_graph(pic_ctx *c);

// Largest displacement (cells) along d in one step: the speed of light, min(1, dt / d_d).
double light_bound(const pic_ctx *c, int d) { return std::min(1.0, c->dt / c->d[d]); }

int make_species(pic_ctx *c, double q, double m, int frozen, int64_t cap, int *sid, bool lattice = false)
{
    drop_graph(c);   // a captured step sequence does not know the new species
    if (c->nsp >= kMaxSpecies) return fail(c, PIC_ERR_ARG, "too many species (max 8)");
    if (cap < 1 || cap >= (int64_t)std::numeric_limits<int>::max() - kChunk)
        return fail(c, PIC_ERR_ARG, "species capacity out of range");
    if (!(m > 0)) return fail(c, PIC_ERR_ARG, "species mass must be > 0");
    Species &s = c->sp[c->nsp];
    s = Species();
    s.q = q;
    s.m = m;
    s.frozen = frozen ? 1 : 0;
    s.cap = cap;
    s.max_items = c->ntiles + cap / kChunkMin + 2;
    int r;
    if (lattice) {
        // a ring of lattice planes replaces the particle records: live planes span the active z
        // range, so plane m - plane_cap is always below the grid when plane m is injected
        s.lattice = 1;
        s.cap = 0;
        s.plane_cap = (int64_t)c->ppc[2] * (c->n[2] + 4) + 2;
        if ((r = alloc_zero(c, &s.planes, s.plane_cap)) || (r = alloc_zero(c, &s.tx, c->n[0])) ||
            (r = alloc_zero(c, &s.ty, c->n[1])) || (r = alloc_zero(c, &s.zacc, c->n[2])) ||
            (r = alloc_zero(c, &s.count, 4)))
            return r;
        CK(cudaMemsetAsync(s.planes, 0xff, sizeof(PlaneRec) * s.plane_cap, c->stream));   // kz = -1: empty
        *sid = c->nsp++;
        return PIC_OK;
    }
    if ((r = alloc_zero(c, &s.pos, cap)) || (r = alloc_zero(c, &s.mom, cap)) || (r = alloc_zero(c, &s.pos2, cap)) ||
        (r = alloc_zero(c, &s.mom2, cap)) || (r = alloc_zero(c, &s.id, cap)) || (r = alloc_zero(c, &s.id2, cap)) ||
        (r = alloc_zero(c, &s.count, 4)) || (r = alloc_zero(c, &s.rank, cap)) ||
        (r = alloc_zero(c, &s.items, s.max_items)) || (r = alloc_zero(c, &s.cell_start, c->n_keys + 1)) ||
        (r = alloc_zero(c, &s.chunk_start, c->ntiles + 1)) || (r = alloc_zero(c, &s.dlim, 4)) ||
        (r = alloc_zero(c, &s.sparse_start, c->ntiles + 1)) || (r = alloc_zero(c, &s.sparse_tiles, c->ntiles)) ||
        (r = alloc_zero(c, &s.tile_start, c->ntiles + 1)) || (r = alloc_zero(c, &s.occ, c->ntiles + 1)) ||
        (r = alloc_zero(c, &s.dmax, 4)))
        return r;
    {
        // the first deposit assumes the speed of light
        const float b[4] = {(float)light_bound(c, 0), (float)light_bound(c, 1), (float)light_bound(c, 2), 0.f};
        CK(cudaMemcpyAsync(s.dlim, b, sizeof(b), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (c->runs > 1) {
        s.wmax_run.assign(c->runs, 0.0);
        if ((r = alloc_zero(c, &s.wrun, (size_t)c->runs))) return r;
    }
    *sid = c->nsp++;
    return PIC_OK;
}

// Upload the per-run largest weights of species s (ensembles).
int upload_wrun(pic_ctx *c, Species &s)
{
    if (!s.wrun) return PIC_OK;
    std::vector<float> w(s.wmax_run.size());
    for (size_t q = 0; q < w.size(); q++) w[q] = (float)s.wmax_run[q];
    CK(cudaMemcpyAsync(s.wrun, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

void set_tiles(pic_ctx *c)
{
    c->ntiles = 1;
    for (int d = 0; d < 3; d++) {
        c->nt[d] = (c->n[d] + c->T[d] - 1) / c->T[d];
        c->ntiles *= c->nt[d];
    }
    c->n_keys = (int64_t)c->ntiles * c->T[0] * c->T[1] * c->T[2] * 8;   // cells x offset octants
}

int alloc_tile_scratch(pic_ctx *c)
{
    if (c->hist_tmp) dfree(c, c->hist_tmp);
    c->hist_tmp_n = scan_scratch_size(std::max<int64_t>(c->n_keys + 1, c->ntiles + 1));
    return alloc_zero(c, &c->hist_tmp, c->hist_tmp_n);
}

double shifts_due(const pic_ctx *c, int64_t n) { return std::floor(c->vw * (double)n * c->dt / c->d[2]); }

// A tile size the particle kernel can run: 2..16 cells per dim, the tile's shared-memory region
// (tile + drift margin + stencil halo) within the shared memory of one CTA, and for an ensemble a
// z size that divides the rows of a run (tiles never straddle runs).
int check_tile(pic_ctx *c, const int T[3], int margin)
{
    for (int d = 0; d < 3; d++)
        if (T[d] < 1 || T[d] > 16) return fail(c, PIC_ERR_ARG, "tile sizes must be 1..16");
    if (margin < 0 || margin > 2) return fail(c, PIC_ERR_ARG, "margin must be 0..2");
    int R3 = 1;
    for (int d = 0; d < 3; d++) R3 *= T[d] + 2 * margin + margin_lo(c) + margin_hi(c);
    if ((size_t)R3 * 12 * sizeof(float) + 40 * 1024 > 224 * 1024)
        return fail(c, PIC_ERR_ARG, "tile region exceeds shared memory");
    if (c->runs > 1 && c->nzr % T[2] != 0)
        return fail(c, PIC_ERR_ARG, "ensemble: the tile's z size must divide the rows of a run");
    return PIC_OK;
}

// Changes the tile size of a context that holds species: the per-species tile tables (sort keys,
// work items, sparse-tile lists) are reallocated for the new tiling and the next step sorts.
int retile(pic_ctx *c, const int T[3])
{
    drop_graph(c);
    for (int d = 0; d < 3; d++) c->T[d] = T[d];
    set_tiles(c);
    int r = alloc_tile_scratch(c);
    if (r) return r;
    for (int si = 0; si < c->nsp; si++) {
        Species &s = c->sp[si];
        if (s.lattice) continue;
        dfree(c, s.items);
        dfree(c, s.cell_start);
        dfree(c, s.chunk_start);
        dfree(c, s.sparse_start);
        dfree(c, s.sparse_tiles);
        dfree(c, s.tile_start);
        dfree(c, s.occ);
        s.items = nullptr;
        s.cell_start = s.chunk_start = s.sparse_start = s.sparse_tiles = s.tile_start = s.occ = nullptr;
        s.max_items = c->ntiles + s.cap / kChunkMin + 2;
        if ((r = alloc_zero(c, &s.items, s.max_items)) || (r = alloc_zero(c, &s.cell_start, c->n_keys + 1)) ||
            (r = alloc_zero(c, &s.chunk_start, c->ntiles + 1)) || (r = alloc_zero(c, &s.sparse_start, c->ntiles + 1)) ||
            (r = alloc_zero(c, &s.sparse_tiles, c->ntiles)) || (r = alloc_zero(c, &s.tile_start, c->ntiles + 1)) ||
            (r = alloc_zero(c, &s.occ, c->ntiles + 1)))
            return r;
    }
    c->sort_base = c->step;   // the stored order is of the old tiles: sort before the next push
    return PIC_OK;
}

// Tracing: a pair of events around a launch group of class cls.
cudaEvent_t take_event(pic_ctx *c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

struct TraceScope {
    pic_ctx *c;
    int cls;
    cudaEvent_t a = nullptr;
    TraceScope(pic_ctx *cc, int k) : c(cc), cls(k) {
        if (c->trace_on && (a = take_event(c))) cudaEventRecord(a, c->stream);
    }
    ~TraceScope() {
        if (!a) return;
        cudaEvent_t b = take_event(c);
        if (!b) { c->ev_pool.push_back(a); return; }
        cudaEventRecord(b, c->stream);
        c->ev_pending.push_back({cls, {a, b}});
    }
};

enum { TR_SORT = 0, TR_PUSH = 1, TR_PUSH_FROZEN = 2, TR_FIELDS = 3, TR_WINDOW = 4, TR_INJECT = 5, TR_OTHER = 6 };

// Particle records of a species for the diagnostics: the species' own, or for a lattice species
// temporary records materialised from its planes, released (after the stream drains) with the view.
struct RecordView {
    pic_ctx *c = nullptr;
    Species s;
    bool tmp = false;
    ~RecordView()
    {
        if (!tmp) return;
        cudaStreamSynchronize(c->stream);
        dfree(c, s.pos);
        dfree(c, s.mom);
        dfree(c, s.id);
        dfree(c, s.count);
    }
};

int record_view(pic_ctx *c, int si, RecordView &v)
{
    v.c = c;
    v.s = c->sp[si];
    if (!v.s.lattice) return PIC_OK;
    v.tmp = true;
    v.s.pos = v.s.mom = nullptr;
    v.s.id = v.s.count = nullptr;
    const int64_t per_plane = (int64_t)(c->xr[1] - c->xr[0]) * (c->xr[3] - c->xr[2]) * c->ppc[0] * c->ppc[1];
    const int64_t n = v.s.plane_cap * per_plane;
    int r;
    if ((r = alloc_zero(c, &v.s.pos, n)) || (r = alloc_zero(c, &v.s.mom, n)) || (r = alloc_zero(c, &v.s.id, n)) ||
        (r = alloc_zero(c, &v.s.count, 4)))
        return r;
    v.s.cap = n;
    CK(launch_lattice_records(c, si, v.s));
    return PIC_OK;
}

int inject_due(pic_ctx *c)
{
    if (c->bc[2][0] == PIC_BC_PERIODIC) return PIC_OK;   // the periodic lattice is filled once
    const int64_t m1 = plane_max(c, c->step, c->shifts);
    if (m1 <= c->m_last) return PIC_OK;
    const int64_t per_plane = (int64_t)(c->xr[1] - c->xr[0]) * (c->xr[3] - c->xr[2]) * c->ppc[0] * c->ppc[1];
    const int64_t add = (m1 - c->m_last) * per_plane;
    for (int si : {c->sp_e, c->sp_i}) {
        Species &s = c->sp[si];
        if (s.lattice) continue;
        if (s.bound + add > s.cap) {
            CK(cudaStreamSynchronize(c->stream));
            int cnt = 0;
            CK(cudaMemcpy(&cnt, s.count, sizeof(int), cudaMemcpyDeviceToHost));
            s.bound = cnt;
            if (s.bound + add > s.cap)
                return fail(c, PIC_ERR_CAPACITY, "plasma species capacity exhausted by injection");
        }
    }
    {
        TraceScope ts(c, TR_INJECT);
        CK(launch_inject(c, c->m_last + 1, m1));
    }
    c->m_last = m1;
    return PIC_OK;
}

ExtDev ext_step(const pic_ctx *c)
{
    ExtDev x{};
    x.type = c->ext_type;
    if (!x.type) return x;
    const double kp = c->ku * c->gR;              // k'_u
    const double tp = (double)c->step * c->dt;
    const double two_pi = 2.0 * M_PI;
    x.B0g = (float)(c->gR * c->B0);
    x.beta_R = (float)c->bR;
    x.kdz = (float)(kp * c->d[2]);
    x.theta = (float)std::fmod(kp * ((double)c->shifts * c->d[2] + c->bR * tp) + c->phase0, two_pi);
    x.phase_tab = c->phase_tab;
    x.amp_tab = c->amp_tab;
    x.kuy = (float)(c->ku * c->d[1]);
    x.y0 = (float)(0.5 * c->n[1]);
    x.igR = (float)(1.0 / c->gR);
    x.clock = c->dclock;
    {
        const double kp = c->ku * c->gR;
        x.th_a = kp * c->bR * c->dt;
        x.th_b = kp * (double)c->shifts * c->d[2] + c->phase0;
    }
    if (std::isfinite(c->z_start) && c->ramp >= 0.0) {
        const double a = c->gR * c->d[2];
        const double b = c->gR * ((double)c->shifts * c->d[2] + c->bR * tp) - c->z_start;
        const double sc = c->ramp > 0.0 ? 1.0 / c->ramp : 1.0;
        x.ramp_mode = c->ramp > 0.0 ? 1 : 2;
        x.ramp_a = (float)(a * sc);
        x.ramp_b = (float)(b * sc);
        x.rb_a = c->gR * c->bR * c->dt * sc;
        x.rb_b = (c->gR * (double)c->shifts * c->d[2] - c->z_start) * sc;
    }
    return x;
}

}  // namespace

namespace gbpic {

GridDev grid_dev(const pic_ctx *c)
{
    GridDev g{};
    for (int d = 0; d < 3; d++) {
        g.n[d] = c->n[d];
        g.periodic[d] = c->bc[d][0] == PIC_BC_PERIODIC;
        g.d[d] = (float)c->d[d];
        g.dt_over_d[d] = (float)(c->dt / c->d[d]);
    }
    g.dt = (float)c->dt;
    g.mlo = margin_lo(c);
    g.mhi = margin_hi(c);
    g.ncell = c->ncell;
    g.cc = c->cc;
    g.nzr = c->nzr;
    return g;
}

TileDev tile_dev(const pic_ctx *c, const Species &s)
{
    TileDev t{};
    for (int d = 0; d < 3; d++) {
        t.T[d] = c->T[d];
        t.nt[d] = c->nt[d];
    }
    t.tile_cells = c->T[0] * c->T[1] * c->T[2];
    t.M = c->M;
    t.hl = margin_lo(c);
    for (int d = 0; d < 3; d++) t.R[d] = c->T[d] + 2 * c->M + margin_lo(c) + margin_hi(c);
    t.cell_start = s.cell_start;
    t.tile_start = s.tile_start;
    t.items = s.items;
    t.sparse_tiles = s.sparse_tiles;
    t.chunk = s.chunk;
    t.cc = c->cc;
    return t;
}

SpeciesDev species_dev(const pic_ctx *c, const Species &s)
{
    SpeciesDev d{};
    d.pos = s.pos;
    d.mom = s.mom;
    d.id = s.id;
    d.count = s.count;
    d.h_qm = (float)(0.5 * s.q / s.m * c->dt);
    const double V = c->d[0] * c->d[1] * c->d[2];
    for (int k = 0; k < 3; k++) {
        d.cf[k] = (float)(-s.q * c->d[k] / (c->dt * V));
        // |contribution| <= |cf| w |prefix DS| |A A + DS DS/12|; |prefix DS| <= |d_k| and
        // |A A + DS DS/12| <= 1.1
        d.jb[k] = (float)(1.1 * std::fabs((double)d.cf[k]));
    }
    d.wmax = (float)s.wmax;
    d.wrun = s.wrun;
    d.dlim = s.dlim;
    d.dmax = s.dmax;
    d.nfall = c->nfall;
    d.pusher = c->pusher;
    d.frozen = s.frozen;
    d.cap = (int)s.cap;
    return d;
}

PmlDev pml_dev(const pic_ctx *c)
{
    PmlDev p{};
    p.on = c->psiE != nullptr;
    if (!p.on) return p;
    for (int d = 0; d < 3; d++) {
        p.bE[d] = c->pml_coef + d * c->nmax;
        p.bB[d] = c->pml_coef + (3 + d) * c->nmax;
    }
    p.psiE = c->psiE;
    p.psiB = c->psiB;
    return p;
}

}  // namespace gbpic

namespace {

int bits_for(int n)
{
    int b = 0;
    while ((1 << b) < n) b++;
    return b;
}

// A context of `runs` independent runs of grid.nz rows each, stacked along z (runs = 1: one run).
int create_impl(pic_ctx **out, int runs, pic_grid grid, const double dx[3], double dt, double gamma_boost,
                const pic_boundaries *bc, int shape_order, const pic_device *dev)
{
    if (!out) return fail(nullptr, PIC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!dx || !bc) return fail(nullptr, PIC_ERR_ARG, "dx and bc are required");
    if (runs < 1 || runs > 4096) return fail(nullptr, PIC_ERR_ARG, "runs must be 1..4096");
    if (grid.nz < 1 || (int64_t)grid.nz * runs > (1 << 20)) return fail(nullptr, PIC_ERR_ARG, "nz * runs must be 1..2^20");
    const int n[3] = {grid.nx, grid.ny, grid.nz * runs};
    if (n[0] < 1 || n[1] < 1 || n[0] > 1024 || n[1] > 1024)
        return fail(nullptr, PIC_ERR_ARG, "nx and ny must be 1..1024 cells");
    if (bits_for(n[0]) + bits_for(n[1]) + bits_for(n[2]) > 31)
        return fail(nullptr, PIC_ERR_ARG, "grid too large: the packed cell index needs more than 31 bits");
    if (runs > 1) {
        if (bc->face[2][0] != PIC_BC_PERIODIC || bc->face[2][1] != PIC_BC_PERIODIC)
            return fail(nullptr, PIC_ERR_ARG, "ensemble runs are stacked along z: z must be periodic");
        if (grid.nz % 8 != 0) return fail(nullptr, PIC_ERR_ARG, "ensemble runs need nz a multiple of the tile size 8");
    }
    if (shape_order != 1 && shape_order != 2) return fail(nullptr, PIC_ERR_ARG, "shape_order must be 1 (CIC) or 2 (TSC)");
    double inv2 = 0;
    for (int d = 0; d < 3; d++) {
        if (!(dx[d] > 0)) return fail(nullptr, PIC_ERR_ARG, "cell sizes must be > 0");
        inv2 += 1.0 / (dx[d] * dx[d]);
    }
    if (!(dt > 0) || !(dt < 1.0 / std::sqrt(inv2))) return fail(nullptr, PIC_ERR_ARG, "dt must satisfy 0 < dt < Courant limit");
    if (!(gamma_boost >= 1.0)) return fail(nullptr, PIC_ERR_ARG, "gamma_boost must be >= 1");
    if ((int64_t)n[0] * n[1] * n[2] * 8 >= ((int64_t)1 << 31) - 4096)
        return fail(nullptr, PIC_ERR_ARG, "grid too large: 8 sort keys per cell must fit in int32");
    bool any_pml = false;
    for (int d = 0; d < 3; d++) {
        for (int f = 0; f < 2; f++) {
            const int b = bc->face[d][f];
            if (b != PIC_BC_PERIODIC && b != PIC_BC_PML && b != PIC_BC_OPEN) return fail(nullptr, PIC_ERR_ARG, "unknown boundary");
            any_pml = any_pml || b == PIC_BC_PML;
        }
        if ((bc->face[d][0] == PIC_BC_PERIODIC) != (bc->face[d][1] == PIC_BC_PERIODIC))
            return fail(nullptr, PIC_ERR_ARG, "a periodic dimension must be periodic on both faces");
        const int need = shape_order == 1 ? 4 : 6;
        if (bc->face[d][0] != PIC_BC_PERIODIC && n[d] < need) return fail(nullptr, PIC_ERR_ARG, "non-periodic dim too small");
    }
    if (any_pml) {
        if (bc->pml_cells < 1) return fail(nullptr, PIC_ERR_ARG, "pml_cells must be >= 1 with a PML face");
        for (int d = 0; d < 3; d++)
            if ((bc->face[d][0] == PIC_BC_PML || bc->face[d][1] == PIC_BC_PML) && 2 * bc->pml_cells >= n[d])
                return fail(nullptr, PIC_ERR_ARG, "PML layers thicker than half the grid");
    }
    if (bc->moving_window) {
        if (bc->face[2][0] == PIC_BC_PERIODIC) return fail(nullptr, PIC_ERR_ARG, "moving window needs a non-periodic z");
        if (!(bc->window_v > 0) || !(bc->window_v * dt < dx[2])) return fail(nullptr, PIC_ERR_ARG, "window_v must give < 1 shift per step");
    }

    pic_ctx *c = new pic_ctx();
    if (dev) c->dev = *dev;
    if (cudaSetDevice(c->dev.device) != cudaSuccess) {
        delete c;
        return fail(nullptr, PIC_ERR_CUDA, "cudaSetDevice failed");
    }
    if (c->dev.stream) {
        c->stream = (cudaStream_t)c->dev.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(nullptr, PIC_ERR_CUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev.device);
    for (int d = 0; d < 3; d++) {
        c->n[d] = n[d];
        c->d[d] = dx[d];
        c->bc[d][0] = bc->face[d][0];
        c->bc[d][1] = bc->face[d][1];
    }
    c->runs = runs;
    c->nzr = grid.nz;
    c->cc.sj = bits_for(n[0]);
    c->cc.sk = c->cc.sj + bits_for(n[1]);
    c->cc.mi = (1 << c->cc.sj) - 1;
    c->cc.mj = (1 << (c->cc.sk - c->cc.sj)) - 1;
    c->dt = dt;
    c->gR = gamma_boost;
    c->bR = std::sqrt(1.0 - 1.0 / (gamma_boost * gamma_boost));
    c->pml = any_pml ? bc->pml_cells : 0;
    c->moving = bc->moving_window ? 1 : 0;
    c->vw = bc->window_v;
    c->order = shape_order;
    c->ncell = (int64_t)n[0] * n[1] * n[2];
    c->nmax = std::max({n[0], n[1], n[2]});
    set_tiles(c);

    auto bail = [&](int r) {
        std::string m = c->msg;
        pic_destroy(c);
        return fail(nullptr, r, m);
    };
    int r;
    if ((r = alloc_zero(c, &c->E, 3 * c->ncell)) || (r = alloc_zero(c, &c->B, 3 * c->ncell)) ||
        (r = alloc_zero(c, &c->J, 3 * c->ncell)) || (r = alloc_zero(c, &c->err, 4)) || (r = alloc_zero(c, &c->nfall, 1)) ||
        (r = alloc_zero(c, &c->dclock, 1)) ||
        (r = alloc_zero(c, &c->work, 2 * kMaxSpecies)) || (r = alloc_zero(c, &c->red, 512 * 16 + 1024)) ||
        (r = alloc_zero(c, &c->shift_tab, 24)) || (r = alloc_tile_scratch(c)))
        return bail(r);
    if (any_pml) {
        if ((r = alloc_zero(c, &c->psiE, 6 * c->ncell)) || (r = alloc_zero(c, &c->psiB, 6 * c->ncell)) ||
            (r = alloc_zero(c, &c->pml_coef, 6 * c->nmax)))
            return bail(r);
        // CPML conductivity: cubic grading over pml_cells, normal reflection 1e-8
        std::vector<float> coef(6 * c->nmax, 1.f);
        const double L = (double)c->pml;
        for (int d = 0; d < 3; d++) {
            const double smax = 4.0 * (-std::log(1e-8)) / (2.0 * L * c->d[d]);
            for (int i = 0; i < n[d]; i++) {
                for (int half = 0; half < 2; half++) {
                    const double pos = i + 0.5 * half;
                    double depth = 0.0;
                    if (c->bc[d][0] == PIC_BC_PML && pos < L) depth = L - pos;
                    if (c->bc[d][1] == PIC_BC_PML && pos > (n[d] - 1) - L) depth = std::max(depth, pos - ((n[d] - 1) - L));
                    const double rr = depth / L;
                    const double sig = depth > 0 ? smax * rr * rr * rr : 0.0;
                    if (half == 0) coef[d * c->nmax + i] = (float)std::exp(-sig * c->dt);
                    else coef[(3 + d) * c->nmax + i] = (float)std::exp(-sig * 0.5 * c->dt);
                }
            }
        }
        // on the context stream, after the zeroing memset (a legacy-stream cudaMemcpy does not wait
        // for a non-blocking stream, and the memset could land after it)
        if (cudaMemcpyAsync(c->pml_coef, coef.data(), coef.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return bail(fail_cuda(c, cudaGetLastError(), "copy PML coefficients"));
    }
    {
        std::vector<float *> tab;
        for (int q = 0; q < 3; q++) {
            tab.push_back(c->E + q * c->ncell);
            tab.push_back(c->B + q * c->ncell);
            tab.push_back(c->J + q * c->ncell);
        }
        if (c->psiE)
            for (int q = 0; q < 6; q++) {
                tab.push_back(c->psiE + q * c->ncell);
                tab.push_back(c->psiB + q * c->ncell);
            }
        c->shift_n = (int)tab.size();
        if (cudaMemcpyAsync(c->shift_tab, tab.data(), tab.size() * sizeof(float *), cudaMemcpyHostToDevice, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return bail(fail_cuda(c, cudaGetLastError(), "copy shift table"));
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(fail_cuda(c, cudaGetLastError(), "create sync"));
    *out = c;
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_create(pic_ctx **out, pic_grid grid, const double dx[3], double dt, double gamma_boost,
               const pic_boundaries *bc, int shape_order, const pic_device *dev)
{
    return create_impl(out, 1, grid, dx, dt, gamma_boost, bc, shape_order, dev);
}

int pic_create_batch(pic_ctx **out, int runs, pic_grid grid, const double dx[3], double dt, double gamma_boost,
                     const pic_boundaries *bc, int shape_order, const pic_device *dev)
{
    return create_impl(out, runs, grid, dx, dt, gamma_boost, bc, shape_order, dev);
}

int pic_set_tuning(pic_ctx *c, const pic_tuning *t)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!t) return fail(c, PIC_ERR_ARG, "tuning is NULL");
    if (c->nsp > 0) return fail(c, PIC_ERR_STATE, "set tuning before creating species");
    if (t->sort_every < 1) return fail(c, PIC_ERR_ARG, "sort_every must be >= 1");
    if ((r = check_tile(c, t->tile, t->margin))) return r;
    for (int d = 0; d < 3; d++) c->T[d] = t->tile[d];
    drop_graph(c);
    c->sort_every = t->sort_every;
    c->M = t->margin;
    set_tiles(c);
    return alloc_tile_scratch(c);
}

}  // extern "C"

namespace {

// Creates a species and loads n_run[r] particles into each run r (arrays run-major, [3][n] with
// n the total).
int load_impl(pic_ctx *c, const pic_species *sp, const int64_t *n_run, int nr, const double *x, const double *u,
              const double *w, int frame, int *species_id)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!sp || !species_id || !n_run) return fail(c, PIC_ERR_ARG, "invalid species arguments");
    int64_t n = 0;
    for (int q = 0; q < nr; q++) {
        if (n_run[q] < 0) return fail(c, PIC_ERR_ARG, "negative particle count");
        n += n_run[q];
    }
    if (n >= (int64_t)std::numeric_limits<int>::max() - kChunk) return fail(c, PIC_ERR_ARG, "too many particles");
    if (n > 0 && (!x || !u)) return fail(c, PIC_ERR_ARG, "x and u are required when n > 0");
    if (frame != PIC_FRAME_LAB && frame != PIC_FRAME_BOOSTED) return fail(c, PIC_ERR_ARG, "unknown frame");
    const int64_t cap = std::max<int64_t>(sp->capacity, std::max<int64_t>(n, 1));
    int sid;
    if ((r = make_species(c, sp->q, sp->m, sp->frozen, cap, &sid))) return r;
    Species &s = c->sp[sid];
    double *dx = nullptr, *du = nullptr, *dw = nullptr;
    if (n > 0) {
        dx = static_cast<double *>(dalloc(c, sizeof(double) * 3 * n));
        du = static_cast<double *>(dalloc(c, sizeof(double) * 3 * n));
        if (w) dw = static_cast<double *>(dalloc(c, sizeof(double) * n));
        if (!dx || !du || (w && !dw)) return fail(c, PIC_ERR_ALLOC, "staging allocation failed");
        CK(cudaMemcpyAsync(dx, x, sizeof(double) * 3 * n, cudaMemcpyDefault, c->stream));
        CK(cudaMemcpyAsync(du, u, sizeof(double) * 3 * n, cudaMemcpyDefault, c->stream));
        if (w) CK(cudaMemcpyAsync(dw, w, sizeof(double) * n, cudaMemcpyDefault, c->stream));
    }
    int64_t off = 0;
    for (int q = 0; q < nr; q++) {
        CK(launch_load(c, sid, n_run[q], dx ? dx + off : nullptr, du ? du + off : nullptr, dw ? dw + off : nullptr,
                       frame, sp->origin, sp->match_undulator, s.next_id + off, q, n));
        off += n_run[q];
    }
    s.next_id += n;
    s.bound += n;
    if (n > 0) {
        double wm = 0;
        CK(species_wmax(c, sid, &wm));
        s.wmax = std::max(s.wmax, wm);
    }
    CK(launch_dlim_from_momenta(c, sid));
    if (c->runs > 1) {
        int64_t o2 = 0;
        for (int q = 0; q < nr; q++) {
            double wm = n_run[q] > 0 ? 1.0 : 0.0;
            if (dw && n_run[q] > 0) CK(absmax_f64(c, dw + o2, n_run[q], &wm));
            s.wmax_run[q] = std::max(s.wmax_run[q], wm);
            o2 += n_run[q];
        }
        if ((r = upload_wrun(c, s))) return r;
    }
    if (n > 0) {
        CK(cudaStreamSynchronize(c->stream));
        dfree(c, dx);
        dfree(c, du);
        dfree(c, dw);
    }
    *species_id = sid;
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_load_species(pic_ctx *c, const pic_species *sp, int64_t n, const double *x, const double *u,
                     const double *w, int frame, int *species_id)
{
    int r = check_ctx(c);
    if (r) return r;
    if (c->runs > 1) return fail(c, PIC_ERR_STATE, "ensemble context: load with pic_load_species_batch");
    return load_impl(c, sp, &n, 1, x, u, w, frame, species_id);
}

int pic_load_species_batch(pic_ctx *c, const pic_species *sp, const int64_t *n_run, const double *x, const double *u,
                           const double *w, int frame, int *species_id)
{
    int r = check_ctx(c);
    if (r) return r;
    return load_impl(c, sp, n_run, c->runs, x, u, w, frame, species_id);
}

int pic_set_external_field(pic_ctx *c, const pic_external *f)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!f) return fail(c, PIC_ERR_ARG, "external field is NULL");
    if (f->type == PIC_EXT_NONE) {
        c->ext_type = 0;
        return PIC_OK;
    }
    if (f->type != PIC_EXT_PLANAR_UNDULATOR && f->type != PIC_EXT_PLANAR_UNDULATOR_3D)
        return fail(c, PIC_ERR_ARG, "unknown external field type");
    if (!(f->lambda_u > 0)) return fail(c, PIC_ERR_ARG, "lambda_u must be > 0");
    drop_graph(c);   // captured launches hold the field's constants
    c->ext_type = f->type;
    c->K = f->K;
    c->lam_u = f->lambda_u;
    c->ku = 2.0 * M_PI / f->lambda_u;
    c->B0 = f->K * c->ku;
    c->phase0 = f->phase;
    c->z_start = f->z_start;
    c->ramp = f->ramp_len;
    if (c->runs > 1 && std::isfinite(f->z_start) && f->ramp_len >= 0.0)
        return fail(c, PIC_ERR_ARG, "ensemble: the undulator must fill the periodic box (no entrance ramp)");
    if (!c->phase_tab && (r = alloc_zero(c, &c->phase_tab, c->n[2]))) return r;
    std::vector<float> tab(c->n[2]);
    const double kdz = c->ku * c->gR * c->d[2];
    // phase of row k in its own run's coordinates (k mod nzr; k for a single run)
    for (int k = 0; k < c->n[2]; k++) tab[k] = (float)std::fmod(kdz * (k % c->nzr), 2.0 * M_PI);
    CK(cudaMemcpyAsync(c->phase_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->B0_run.clear();
    return PIC_OK;
}

int pic_set_external_field_batch(pic_ctx *c, const pic_external *f)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!f) return fail(c, PIC_ERR_ARG, "external field is NULL");
    for (int q = 1; q < c->runs; q++)
        if (f[q].type != f[0].type || f[q].lambda_u != f[0].lambda_u || f[q].phase != f[0].phase ||
            f[q].z_start != f[0].z_start || f[q].ramp_len != f[0].ramp_len)
            return fail(c, PIC_ERR_ARG, "ensemble runs may differ in K only");
    if ((r = pic_set_external_field(c, &f[0]))) return r;
    if (f[0].type == PIC_EXT_NONE) return PIC_OK;
    c->B0_run.resize(c->runs);
    for (int q = 0; q < c->runs; q++) c->B0_run[q] = f[q].K * c->ku;
    if (!c->amp_tab && (r = alloc_zero(c, &c->amp_tab, c->n[2]))) return r;
    std::vector<float> amp(c->n[2]);
    for (int k = 0; k < c->n[2]; k++) amp[k] = (float)(c->gR * c->B0_run[k / c->nzr]);
    CK(cudaMemcpyAsync(c->amp_tab, amp.data(), amp.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

}  // extern "C"

namespace {

// Background plasma; scale: density factor of each run (ensembles) or NULL.
int plasma_impl(pic_ctx *c, const pic_plasma *p, const double *scale, int *electron_id, int *ion_id)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!p || !electron_id || !ion_id) return fail(c, PIC_ERR_ARG, "plasma arguments are NULL");
    if (c->plasma) return fail(c, PIC_ERR_STATE, "plasma already set");
    for (int d = 0; d < 3; d++)
        if (p->ppc[d] < 1 || p->ppc[d] > 16) return fail(c, PIC_ERR_ARG, "ppc must be 1..16 per dim");
    if (p->x_range[0] < 0 || p->x_range[1] > c->n[0] || p->x_range[0] >= p->x_range[1] || p->x_range[2] < 0 ||
        p->x_range[3] > c->n[1] || p->x_range[2] >= p->x_range[3])
        return fail(c, PIC_ERR_ARG, "x_range outside the grid");
    if (p->n_nodes < 1 || !p->z_nodes || !p->density) return fail(c, PIC_ERR_ARG, "density profile required");
    for (int d = 0; d < 3; d++) c->ppc[d] = p->ppc[d];
    for (int k = 0; k < 4; k++) c->xr[k] = p->x_range[k];
    const int64_t per_plane = (int64_t)(c->xr[1] - c->xr[0]) * (c->xr[3] - c->xr[2]) * c->ppc[0] * c->ppc[1];
    int64_t cap = p->capacity;
    if (cap <= 0) {
        const double planes_window = (double)c->n[2] * c->ppc[2] + 2;
        const double rate = c->ppc[2] * (c->bR + c->vw) * c->dt / c->d[2] + 1e-9;
        cap = (int64_t)(per_plane * (planes_window + rate * (c->sort_every + 2) * 2 + 8));
    }
    int se, si;
    if ((r = make_species(c, -1.0, 1.0, 0, cap, &se))) return r;
    if ((r = make_species(c, 1.0, 1836.15267343, 1, cap, &si, true))) return r;
    c->nprof = p->n_nodes;
    c->prof_z.assign(p->z_nodes, p->z_nodes + p->n_nodes);
    c->prof_n.assign(p->density, p->density + p->n_nodes);
    if ((r = alloc_zero(c, &c->prof, 2 * (size_t)p->n_nodes))) return r;
    std::vector<double> pr(2 * p->n_nodes);
    for (int i = 0; i < p->n_nodes; i++) {
        pr[i] = p->z_nodes[i];
        pr[p->n_nodes + i] = p->density[i];
    }
    CK(cudaMemcpyAsync(c->prof, pr.data(), pr.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->plasma = 1;
    c->sp_e = se;
    c->sp_i = si;
    if (c->runs > 1) {
        c->dens_run.assign(c->runs, 1.0);
        if (scale)
            for (int q = 0; q < c->runs; q++) {
                if (!(scale[q] >= 0.0)) return fail(c, PIC_ERR_ARG, "density scales must be >= 0");
                c->dens_run[q] = scale[q];
            }
        if ((r = alloc_zero(c, &c->dens_scale, (size_t)c->runs))) return r;
        CK(cudaMemcpyAsync(c->dens_scale, c->dens_run.data(), sizeof(double) * c->runs, cudaMemcpyHostToDevice, c->stream));
    }
    {
        double nmax = 0;
        for (int i = 0; i < p->n_nodes; i++) nmax = std::max(nmax, std::fabs(p->density[i]));
        const double wm1 = c->gR * nmax * c->d[0] * c->d[1] * c->d[2] / ((double)c->ppc[0] * c->ppc[1] * c->ppc[2]);
        double wm = wm1;
        if (c->runs > 1) {
            wm *= *std::max_element(c->dens_run.begin(), c->dens_run.end());
            for (int q = 0; q < c->runs; q++) c->sp[se].wmax_run[q] = wm1 * c->dens_run[q];
            if ((r = upload_wrun(c, c->sp[se]))) return r;
        }
        c->sp[se].wmax = c->sp[si].wmax = wm;
    }
    CK(launch_lattice_profiles(c, si));
    // open z: fill the window between the margins, later planes enter at the front; periodic z:
    // the lattice fills the whole box once and drifts around it (no plane is ever injected)
    const bool zper = c->bc[2][0] == PIC_BC_PERIODIC;
    const double lo = (double)margin_lo(c) + (double)c->shifts + c->bR * (double)c->step * c->dt / c->d[2];
    const int64_t m0 = zper ? 0 : (int64_t)std::ceil((double)c->ppc[2] * lo - 0.5);
    const int64_t m1 = zper ? (int64_t)c->ppc[2] * c->n[2] - 1 : plane_max(c, c->step, c->shifts);
    if ((m1 - m0 + 1) * per_plane > cap) return fail(c, PIC_ERR_CAPACITY, "plasma capacity below the window fill");
    if (m1 - m0 + 1 > c->sp[si].plane_cap) return fail(c, PIC_ERR_CAPACITY, "plasma lattice ring below the window fill");
    if (c->sp[si].plane_cap * per_plane >= (int64_t)std::numeric_limits<int>::max())
        return fail(c, PIC_ERR_ARG, "plasma lattice too large for 32-bit particle slots");
    CK(launch_inject(c, m0, m1));
    CK(launch_dlim_from_momenta(c, se));
    c->m_last = m1;
    CK(cudaStreamSynchronize(c->stream));
    *electron_id = se;
    *ion_id = si;
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_set_plasma(pic_ctx *c, const pic_plasma *p, int *electron_id, int *ion_id)
{
    return plasma_impl(c, p, nullptr, electron_id, ion_id);
}

int pic_set_plasma_batch(pic_ctx *c, const pic_plasma *p, const double *density_scale, int *electron_id, int *ion_id)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!density_scale) return fail(c, PIC_ERR_ARG, "density_scale is NULL");
    return plasma_impl(c, p, density_scale, electron_id, ion_id);
}

}  // extern "C"

namespace {

__global__ void k_tick(long long *clock) { *clock += 1; }

int save_state(pic_ctx *c, StateSnap &st, bool alloc, bool quick = false);
int ad_checkpoint_due(pic_ctx *c);

// One step of the method (the body of pic_step).
int step_once(pic_ctx *c)
{
    int r;
    if ((r = ad_checkpoint_due(c))) return r;
    // the adjoint records sort at every checkpoint, so a recomputed segment repeats its sorts
    const bool ad_sort = c->ad_on && (c->step - c->ad_step0) % c->ad_every == 0;
    const bool sorted = ad_sort || (c->step - c->sort_base) % c->sort_every == 0;
    if (sorted) {
        TraceScope ts(c, TR_SORT);
        for (int si = 0; si < c->nsp; si++)
            if (!c->sp[si].lattice) CK(launch_sort(c, si));
    }
    if (c->ad_rec_n >= 0) {
        if (c->ad_rec_n >= (int)c->ad_rec.size()) return fail(c, PIC_ERR_STATE, "adjoint record overflow");
        StateSnap &st = c->ad_rec[c->ad_rec_n++];
        if (!st.E && (r = save_state(c, st, true))) return r;   // first use allocates (and syncs)
        if ((r = save_state(c, st, false, true))) return r;
        st.sorted = sorted;
    }
    // the lattice species writes J_z whole, before the other species add to it
    const bool lat = c->plasma && c->sp[c->sp_i].lattice;
    CK(cudaMemsetAsync(c->J, 0, sizeof(float) * (lat ? 2 : 3) * c->ncell, c->stream));
    CK(cudaMemsetAsync(c->work, 0, sizeof(int) * 2 * kMaxSpecies, c->stream));
    if (lat) {
        TraceScope ts(c, TR_PUSH_FROZEN);
        CK(launch_lattice_step(c, c->sp_i));
    }
    const ExtDev ext = ext_step(c);
    for (int si = 0; si < c->nsp; si++) {
        if (c->sp[si].lattice) continue;
        TraceScope ts(c, c->sp[si].frozen ? TR_PUSH_FROZEN : TR_PUSH);
        CK(launch_push(c, si, ext));
    }
    if (c->snap) {
        TraceScope ts(c, TR_OTHER);
        CK(launch_snap_record(c));
    }
    if (c->ion_G) {
        // the fading artificial ions' current, averaged over the part of the ramp this step covers
        const double t0 = (double)c->step * c->dt, t1 = t0 + c->dt;
        const double a = std::max(t0, c->ion_t0), b = std::min(t1, c->ion_t0 + c->ion_T);
        if (b > a) {
            TraceScope ts(c, TR_OTHER);
            CK(launch_ion_current(c, (float)((b - a) / (c->ion_T * c->dt))));
        }
    }
    {
        TraceScope ts(c, TR_FIELDS);
        CK(launch_fdtd_b(c, (float)(0.5 * c->dt)));
        CK(launch_fdtd_e(c));
        CK(launch_fdtd_b(c, (float)(0.5 * c->dt)));
    }
    k_tick<<<1, 1, 0, c->stream>>>(c->dclock);
    CK(cudaGetLastError());
    c->kernels++;
    c->step++;
    if (c->moving) {
        const int64_t due = (int64_t)shifts_due(c, c->step);
        while (c->shifts < due) {
            TraceScope ts(c, TR_WINDOW);
            CK(launch_shift_fields(c));
            for (int si = 0; si < c->nsp; si++)
                CK(c->sp[si].lattice ? launch_lattice_shift(c, si) : launch_shift_particles(c, si));
            if (c->ion_G) CK(launch_ion_shift(c));
            c->shifts++;
        }
    }
    if (c->plasma && (r = inject_due(c))) return r;
    return PIC_OK;
}

// A step sequence can be captured once and replayed when nothing the host decides per step
// changes between periods: no moving window, no plasma injection (periodic z), tracing off.
bool graph_eligible(const pic_ctx *c)
{
    if (!c->use_graphs || c->moving || c->trace_on || c->nsp == 0 || c->ad_on || c->ion_G || c->snap) return false;
    if (c->plasma && c->bc[2][0] != PIC_BC_PERIODIC) return false;
    return true;
}

void drop_graph(pic_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_steps = 0;
    c->graph_key = nullptr;
}

const void *pointer_key(const pic_ctx *c)
{
    for (int si = 0; si < c->nsp; si++)
        if (!c->sp[si].lattice) return c->sp[si].pos;
    return nullptr;
}

// ------------------------------------------------------------------ adjoint state

void free_state(pic_ctx *c, StateSnap &st)
{
    dfree(c, st.E);
    dfree(c, st.B);
    for (auto &q : st.sp) {
        dfree(c, q.pos);
        dfree(c, q.mom);
        dfree(c, q.id);
        dfree(c, q.planes);
        dfree(c, q.dcount);
    }
    st = StateSnap();
}

// Copy the run's state (fields E, B; every species' records, counts, displacement bounds and
// lattice planes) into st, allocating its buffers first when alloc (or when st is empty).
// quick: a recorded step (no host synchronisation; counts stay on the device until
// finish_records reads them).
int save_state(pic_ctx *c, StateSnap &st, bool alloc, bool quick)
{
    const size_t f3 = sizeof(float) * 3 * (size_t)c->ncell;
    if (alloc || !st.E) {
        free_state(c, st);
        st.E = static_cast<float *>(dalloc(c, f3));
        st.B = static_cast<float *>(dalloc(c, f3));
        if (!st.E || !st.B) return fail(c, PIC_ERR_ALLOC, "adjoint state allocation failed");
        st.sp.assign(c->nsp, SpeciesSnap());
        for (int si = 0; si < c->nsp; si++) {
            const Species &s = c->sp[si];
            SpeciesSnap &q = st.sp[si];
            if (s.lattice) {
                q.planes = static_cast<PlaneRec *>(dalloc(c, sizeof(PlaneRec) * s.plane_cap));
                if (!q.planes) return fail(c, PIC_ERR_ALLOC, "adjoint state allocation failed");
                continue;
            }
            q.pos = static_cast<float4 *>(dalloc(c, sizeof(float4) * s.cap));
            q.mom = static_cast<float4 *>(dalloc(c, sizeof(float4) * s.cap));
            q.id = static_cast<int *>(dalloc(c, sizeof(int) * s.cap));
            q.dcount = static_cast<int *>(dalloc(c, sizeof(int) * 4));
            if (!q.pos || !q.mom || !q.id || !q.dcount) return fail(c, PIC_ERR_ALLOC, "adjoint state allocation failed");
        }
    }
    st.step = c->step;
    CK(cudaMemcpyAsync(st.E, c->E, f3, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(st.B, c->B, f3, cudaMemcpyDeviceToDevice, c->stream));
    for (int si = 0; si < c->nsp; si++) {
        const Species &s = c->sp[si];
        SpeciesSnap &q = st.sp[si];
        if (s.lattice) {
            CK(cudaMemcpyAsync(q.planes, s.planes, sizeof(PlaneRec) * s.plane_cap, cudaMemcpyDeviceToDevice, c->stream));
            continue;
        }
        // the host bound of the slots in use sizes the copy (no injection in the differentiated
        // runs); q.n becomes the device count once the copies are done
        const size_t nb = (size_t)std::min<int64_t>(s.bound, s.cap);
        if (quick) {
            CK(cudaMemcpyAsync(q.dcount, s.count, sizeof(int) * 4, cudaMemcpyDeviceToDevice, c->stream));
        } else {
            CK(cudaMemcpyAsync(q.count, s.count, sizeof(int) * 4, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(q.dlim, s.dlim, sizeof(float) * 4, cudaMemcpyDeviceToHost, c->stream));
        }
        CK(cudaMemcpyAsync(q.pos, s.pos, sizeof(float4) * nb, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(q.mom, s.mom, sizeof(float4) * nb, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(q.id, s.id, sizeof(int) * nb, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (quick) return PIC_OK;
    CK(cudaStreamSynchronize(c->stream));
    for (int si = 0; si < c->nsp; si++)
        if (!c->sp[si].lattice) st.sp[si].n = st.sp[si].count[0];
    return PIC_OK;
}

// After a segment is recomputed: the recorded steps' particle counts, read once.
int finish_records(pic_ctx *c, int nrec)
{
    for (int k = 0; k < nrec; k++)
        for (int si = 0; si < c->nsp; si++)
            if (!c->sp[si].lattice)
                CK(cudaMemcpyAsync(c->ad_rec[k].sp[si].count, c->ad_rec[k].sp[si].dcount, sizeof(int) * 4,
                                   cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < nrec; k++)
        for (int si = 0; si < c->nsp; si++)
            if (!c->sp[si].lattice) c->ad_rec[k].sp[si].n = c->ad_rec[k].sp[si].count[0];
    return PIC_OK;
}

int restore_state(pic_ctx *c, const StateSnap &st)
{
    const size_t f3 = sizeof(float) * 3 * (size_t)c->ncell;
    CK(cudaMemcpyAsync(c->E, st.E, f3, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->B, st.B, f3, cudaMemcpyDeviceToDevice, c->stream));
    for (int si = 0; si < c->nsp; si++) {
        Species &s = c->sp[si];
        const SpeciesSnap &q = st.sp[si];
        if (s.lattice) {
            CK(cudaMemcpyAsync(s.planes, q.planes, sizeof(PlaneRec) * s.plane_cap, cudaMemcpyDeviceToDevice, c->stream));
            continue;
        }
        CK(cudaMemcpyAsync(s.pos, q.pos, sizeof(float4) * q.n, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(s.mom, q.mom, sizeof(float4) * q.n, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(s.id, q.id, sizeof(int) * q.n, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(s.count, q.count, sizeof(int) * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(s.dlim, q.dlim, sizeof(float) * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemsetAsync(s.dmax, 0, sizeof(unsigned) * 4, c->stream));
    }
    const long long clk = st.step;
    CK(cudaMemcpyAsync(c->dclock, &clk, sizeof(clk), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->step = st.step;
    return PIC_OK;
}

// While recording for the adjoint, a checkpoint is saved at the start of every ad_every-th step.
int ad_checkpoint_due(pic_ctx *c)
{
    if (!c->ad_on || c->ad_rec_n >= 0) return PIC_OK;
    const int64_t rel = c->step - c->ad_step0;
    if (rel < 0 || rel % c->ad_every) return PIC_OK;
    const size_t j = (size_t)(rel / c->ad_every);
    if (j < c->ad_ckpt.size()) return PIC_OK;
    c->ad_ckpt.emplace_back();
    return save_state(c, c->ad_ckpt.back(), true);
}

// Captures `period` steps (two sort periods: every sort swaps the particle buffers, so after two
// the buffers the graph's kernels address are current again) without executing them; the host
// state the capture advanced is restored.
// If capturing fails the context falls back to launching every step (graphs off) and stays usable.
void capture_graph(pic_ctx *c, int64_t period)
{
    drop_graph(c);
    const int64_t step0 = c->step, kern0 = c->kernels;
    const bool poisoned0 = c->poisoned;
    const std::string msg0 = c->msg;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        c->use_graphs = 0;
        return;
    }
    int r = PIC_OK;
    for (int64_t k = 0; k < period && r == PIC_OK; k++) r = step_once(c);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->step = step0;
    const int64_t captured = c->kernels - kern0;
    c->kernels = kern0;
    cudaGraphExec_t x = nullptr;
    if (r == PIC_OK && e == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) == cudaSuccess) {
        c->graph = x;
        c->graph_steps = period;
        c->graph_kernels = captured;
        c->graph_key = pointer_key(c);
    } else {
        cudaGetLastError();
        c->poisoned = poisoned0;
        c->msg = msg0;
        c->use_graphs = 0;
    }
    if (g) cudaGraphDestroy(g);
}

}  // namespace

extern "C" {

int pic_step(pic_ctx *c, int64_t nsteps)
{
    int r = check_ctx(c);
    if (r) return r;
    if (nsteps < 0) return fail(c, PIC_ERR_ARG, "negative step count");
    const int64_t period = 2 * (int64_t)c->sort_every;
    int64_t left = nsteps;
    while (left > 0) {
        const bool at_start = (c->step - c->sort_base) % period == 0;
        if (graph_eligible(c) && at_start && left >= period) {
            if (!c->graph || c->graph_steps != period || c->graph_key != pointer_key(c)) capture_graph(c, period);
            if (c->graph && c->graph_key == pointer_key(c)) {
                CK(cudaGraphLaunch(c->graph, c->stream));
                c->step += period;
                c->kernels += c->graph_kernels;
                left -= period;
                continue;
            }
        }
        if ((r = step_once(c))) return r;
        left--;
    }
    return PIC_OK;
}

int pic_set_pusher(pic_ctx *c, int pusher)
{
    int r = check_ctx(c);
    if (r) return r;
    if (pusher != PIC_PUSHER_BORIS && pusher != PIC_PUSHER_VAY) return fail(c, PIC_ERR_ARG, "unknown pusher");
    if (c->ad_on && pusher != PIC_PUSHER_BORIS) return fail(c, PIC_ERR_STATE, "the adjoint reverses the Boris push");
    drop_graph(c);   // captured launches hold the species parameters
    c->pusher = pusher;
    return PIC_OK;
}

int pic_set_ion_ramp(pic_ctx *c, int species_id, double T_ion)
{
    int r = check_ctx(c);
    if (r) return r;
    if (species_id < 0 || species_id >= c->nsp) return fail(c, PIC_ERR_ARG, "no such species");
    if (c->ad_on) return fail(c, PIC_ERR_STATE, "the adjoint does not differentiate the artificial ions");
    drop_graph(c);
    if (!(T_ion > 0.0)) {
        dfree(c, c->ion_G);
        c->ion_G = nullptr;
        return PIC_OK;
    }
    if (!c->ion_G && (r = alloc_zero(c, &c->ion_G, c->ncell))) return r;
    if (!c->rho && (r = alloc_zero(c, &c->rho, c->ncell))) return r;
    CK(cudaMemsetAsync(c->rho, 0, sizeof(float) * c->ncell, c->stream));
    {
        RecordView v;
        if ((r = record_view(c, species_id, v))) return r;
        CK(launch_rho(c, v.s, c->rho));
    }
    CK(launch_ion_prefix(c, c->rho, c->ion_G));
    CK(cudaStreamSynchronize(c->stream));
    c->ion_t0 = (double)c->step * c->dt;
    c->ion_T = T_ion;
    return PIC_OK;
}

int pic_lab_snapshot(pic_ctx *c, int species_id, double t_lab)
{
    int r = check_ctx(c);
    if (r) return r;
    drop_graph(c);
    dfree(c, c->snap);
    dfree(c, c->snap_state);
    c->snap = nullptr;
    c->snap_state = nullptr;
    c->snap_n = 0;
    c->snap_sp = -1;
    if (std::isnan(t_lab)) return PIC_OK;
    if (species_id < 0 || species_id >= c->nsp || c->sp[species_id].lattice)
        return fail(c, PIC_ERR_ARG, "no such particle species");
    if (c->runs != 1) return fail(c, PIC_ERR_ARG, "the lab snapshot is for a single run");
    const int64_t n = std::max<int64_t>(c->sp[species_id].next_id, 1);
    if ((r = alloc_zero(c, &c->snap, 7 * (size_t)n)) || (r = alloc_zero(c, &c->snap_state, (size_t)n))) return r;
    c->snap_sp = species_id;
    c->snap_n = c->sp[species_id].next_id;
    c->snap_T = t_lab;
    CK(launch_snap_arm(c));
    return PIC_OK;
}

int pic_lab_snapshot_read(pic_ctx *c, double *rec, uint8_t *state, int64_t n, int64_t *n_ids, int64_t *recorded)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!c->snap) return fail(c, PIC_ERR_STATE, "no lab snapshot is armed");
    if (n_ids) *n_ids = c->snap_n;
    if ((rec || state) && n < c->snap_n) return fail(c, PIC_ERR_ARG, "buffers smaller than the snapshot's ids");
    std::vector<uint8_t> st((size_t)std::max<int64_t>(c->snap_n, 1));
    CK(cudaMemcpyAsync(st.data(), c->snap_state, (size_t)c->snap_n, cudaMemcpyDeviceToHost, c->stream));
    if (rec) CK(cudaMemcpyAsync(rec, c->snap, sizeof(double) * 7 * (size_t)c->snap_n, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (state) std::memcpy(state, st.data(), (size_t)c->snap_n);
    if (recorded) {
        int64_t m = 0;
        for (int64_t i = 0; i < c->snap_n; i++) m += st[(size_t)i] == 1;
        *recorded = m;
    }
    return PIC_OK;
}

int pic_lab_snapshot_moments(pic_ctx *c, double k_bunch, pic_moments *out)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!out) return fail(c, PIC_ERR_ARG, "out is NULL");
    if (!c->snap) return fail(c, PIC_ERR_STATE, "no lab snapshot is armed");
    double v[20];
    CK(launch_snap_moments(c, k_bunch, v));
    std::memcpy(out, v, sizeof(v));
    return PIC_OK;
}

int pic_set_gather(pic_ctx *c, int gather)
{
    int r = check_ctx(c);
    if (r) return r;
    if (gather != PIC_GATHER_MOMENTUM && gather != PIC_GATHER_ENERGY) return fail(c, PIC_ERR_ARG, "unknown gather scheme");
    if (c->ad_on && gather != PIC_GATHER_MOMENTUM)
        return fail(c, PIC_ERR_STATE, "the adjoint reverses the momentum-conserving gather");
    drop_graph(c);   // captured launches hold the kernel variant
    c->gather = gather;
    return PIC_OK;
}

int pic_resolution_factor(const pic_ctx *c, double lambda_lab, double *r_rf, int *ok)
{
    if (!c || !r_rf) return PIC_ERR_ARG;
    // sqrt((1 - beta)/(1 + beta)) = 1 / (gamma (1 + beta)), free of cancellation at large gamma
    *r_rf = 8.0 * c->d[2] / (c->gR * (1.0 + c->bR));
    if (ok) *ok = *r_rf < lambda_lab ? 1 : 0;
    return PIC_OK;
}

int pic_resonant_wavenumber(double K, double lambda_u, double gamma_B, double gamma_R, int frame, double *k)
{
    if (!k) return fail(nullptr, PIC_ERR_ARG, "pic_resonant_wavenumber: k is NULL");
    if (!(lambda_u > 0.0) || !(gamma_B >= 1.0) || !(gamma_R >= 1.0) || !(K >= 0.0) || !std::isfinite(K) ||
        !std::isfinite(lambda_u) || !std::isfinite(gamma_B) || !std::isfinite(gamma_R)) {
        return fail(nullptr, PIC_ERR_ARG,
                    "pic_resonant_wavenumber: need lambda_u > 0, K >= 0, gamma_B >= 1, gamma_R >= 1 (finite)");
    }
    if (frame != PIC_FRAME_LAB && frame != PIC_FRAME_BOOSTED) {
        return fail(nullptr, PIC_ERR_ARG, "pic_resonant_wavenumber: frame must be PIC_FRAME_LAB or PIC_FRAME_BOOSTED");
    }
    const double a = 1.0 + 0.5 * K * K;
    // Eq. RadLambda: lambda_l = lambda_u (1 + K^2/2) / (2 gamma_B^2)
    const double k_lab = 2.0 * M_PI * 2.0 * gamma_B * gamma_B / (lambda_u * a);
    if (frame == PIC_FRAME_LAB) { *k = k_lab; return PIC_OK; }
    // a structure moving with the beam's mean lab velocity beta_z (1 - beta_z = a / (2 gamma_B^2))
    // has k' = gamma_R (1 - beta_z beta_R) k in the frame moving at beta_R; the factor is formed
    // as (1 - beta_R) + beta_R (1 - beta_z) with 1 - beta_R = 1 / (gamma_R^2 (1 + beta_R))
    const double bR = std::sqrt(1.0 - 1.0 / (gamma_R * gamma_R));
    const double one_m_bR = 1.0 / (gamma_R * gamma_R * (1.0 + bR));
    const double one_m_bz = a / (2.0 * gamma_B * gamma_B);
    *k = k_lab * gamma_R * (one_m_bR + bR * one_m_bz);
    return PIC_OK;
}

int pic_autotune_tiles(pic_ctx *c, const int *tiles, int n_tiles, int max_sort_every, int *tile_out,
                       int *sort_every_out)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!tiles || n_tiles < 1) return fail(c, PIC_ERR_ARG, "no tile candidates");
    if (max_sort_every < 1) return fail(c, PIC_ERR_ARG, "max_sort_every must be >= 1");
    if (c->ad_on) return fail(c, PIC_ERR_STATE, "the tile cannot change while adjoint checkpoints are recorded");
    for (int q = 0; q < n_tiles; q++)
        if ((r = check_tile(c, tiles + 3 * q, c->M))) return r;
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(c, PIC_ERR_CUDA, "cudaEventCreate failed");
    }
    // every candidate, in two passes (ascending then descending), over whole periods of the
    // current sort cadence (>= 32 steps), each trial starting with a sort on the new tiles
    const int se = c->sort_every;
    const int64_t steps = ((std::max(32, se) + se - 1) / se) * (int64_t)se;
    std::vector<double> tot(n_tiles, 0.0);
    for (int pass = 0; pass < 2 && !r; pass++) {
        for (int q0 = 0; q0 < n_tiles && !r; q0++) {
            const int q = pass == 0 ? q0 : n_tiles - 1 - q0;
            if ((r = retile(c, tiles + 3 * q))) break;
            cudaEventRecord(a, c->stream);
            r = pic_step(c, steps);
            cudaEventRecord(b, c->stream);
            if (r) break;
            float ms = 0;
            if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
                r = fail_cuda(c, cudaGetLastError(), "autotune timing");
                break;
            }
            tot[q] += ms / (double)steps;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r) return r;
    // the first candidate is the reference: another must beat the best so far by 2 %
    int best = 0;
    for (int q = 1; q < n_tiles; q++)
        if (tot[q] < 0.98 * tot[best]) best = q;
    if ((r = retile(c, tiles + 3 * best))) return r;
    int se_best = c->sort_every;
    if ((r = pic_autotune(c, max_sort_every, &se_best))) return r;
    if (tile_out)
        for (int d = 0; d < 3; d++) tile_out[d] = c->T[d];
    if (sort_every_out) *sort_every_out = se_best;
    return PIC_OK;
}

int pic_use_graphs(pic_ctx *c, int on)
{
    int r = check_ctx(c);
    if (r) return r;
    c->use_graphs = on ? 1 : 0;
    if (!on) drop_graph(c);
    return PIC_OK;
}

int pic_autotune(pic_ctx *c, int max_sort_every, int *sort_every_out)
{
    int r = check_ctx(c);
    if (r) return r;
    if (max_sort_every < 1) return fail(c, PIC_ERR_ARG, "max_sort_every must be >= 1");
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(c, PIC_ERR_CUDA, "cudaEventCreate failed");
    }
    std::vector<int> cand;
    for (int se : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32})
        if (se <= max_sort_every) cand.push_back(se);
    // two passes, ascending then descending, so that a cost that drifts as the run evolves
    // weighs on every candidate alike
    std::vector<double> tot(cand.size(), 0.0);
    const int nc = (int)cand.size();
    for (int pass = 0; pass < 2 && !r; pass++) {
        for (int q = 0; q < nc; q++) {
            const int idx = pass == 0 ? q : nc - 1 - q;
            const int se = cand[idx];
            // each trial starts right after a sort and covers whole sort periods (>= 32 steps, so
            // that rare costly steps such as a window shift average out)
            const int64_t steps = ((std::max(32, se) + se - 1) / se) * (int64_t)se;
            c->sort_every = se;
            c->sort_base = c->step;   // the trial's first step sorts
            cudaEventRecord(a, c->stream);
            r = pic_step(c, steps);
            cudaEventRecord(b, c->stream);
            if (r) break;
            float ms = 0;
            if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
                r = fail_cuda(c, cudaGetLastError(), "autotune timing");
                break;
            }
            tot[idx] += ms / (double)steps;
        }
    }
    double best_ms = 0;
    int best = c->sort_every;
    for (int q = 0; q < nc && !r; q++) {
        // a rarer sort must beat the best so far by 2 % (timing noise; fresher sorting is safer)
        if (best_ms == 0 || tot[q] < 0.98 * best_ms) {
            best_ms = tot[q];
            best = cand[q];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (r) return r;
    c->sort_every = best;
    if (sort_every_out) *sort_every_out = best;
    return PIC_OK;
}

int pic_sync(pic_ctx *c)
{
    if (!c) return PIC_ERR_ARG;
    if (c->poisoned) return PIC_ERR_STATE;
    CK(cudaStreamSynchronize(c->stream));
    int e = 0;
    CK(cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        char hex[16];
        std::snprintf(hex, sizeof(hex), "0x%x", (unsigned)e);
        std::string m = std::string("device error word ") + hex + ":";
        if (e & ERR_INDEX) m += " stencil node outside a non-periodic grid;";
        if (e & ERR_CAPACITY) m += " species capacity exceeded;";
        if (e & ERR_MOVE) m += " particle moved one cell or more in a step;";
        if (e & ERR_NAN) m += " non-finite momentum;";
        return fail(c, PIC_ERR_DEVICE, m);
    }
    return PIC_OK;
}

int pic_sort(pic_ctx *c)
{
    int r = check_ctx(c);
    if (r) return r;
    TraceScope ts(c, TR_SORT);
    for (int si = 0; si < c->nsp; si++)
        if (!c->sp[si].lattice) CK(launch_sort(c, si));
    return PIC_OK;
}

int pic_get_fields(pic_ctx *c, int which, float *dst, size_t n)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!dst || n < (size_t)c->ncell) return fail(c, PIC_ERR_ARG, "destination smaller than the grid");
    const float *src = nullptr;
    if (which >= PIC_EX && which <= PIC_EZ) src = c->E + (which - PIC_EX) * c->ncell;
    else if (which >= PIC_BX && which <= PIC_BZ) src = c->B + (which - PIC_BX) * c->ncell;
    else if (which >= PIC_JX && which <= PIC_JZ) src = c->J + (which - PIC_JX) * c->ncell;
    else if (which == PIC_RHO) {
        if (!c->rho && (r = alloc_zero(c, &c->rho, c->ncell))) return r;
        CK(cudaMemsetAsync(c->rho, 0, sizeof(float) * c->ncell, c->stream));
        for (int si = 0; si < c->nsp; si++) {
            RecordView v;
            if ((r = record_view(c, si, v))) return r;
            CK(launch_rho(c, v.s, c->rho));
        }
        src = c->rho;
    } else {
        return fail(c, PIC_ERR_ARG, "unknown field");
    }
    CK(cudaMemcpyAsync(dst, src, sizeof(float) * c->ncell, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

int pic_set_fields(pic_ctx *c, int which, const float *src, size_t n)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!src || n < (size_t)c->ncell) return fail(c, PIC_ERR_ARG, "source smaller than the grid");
    float *dst = nullptr;
    if (which >= PIC_EX && which <= PIC_EZ) dst = c->E + (which - PIC_EX) * c->ncell;
    else if (which >= PIC_BX && which <= PIC_BZ) dst = c->B + (which - PIC_BX) * c->ncell;
    else if (which >= PIC_JX && which <= PIC_JZ) dst = c->J + (which - PIC_JX) * c->ncell;
    else return fail(c, PIC_ERR_ARG, "unknown field");
    CK(cudaMemcpyAsync(dst, src, sizeof(float) * c->ncell, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

int pic_get_particles(pic_ctx *c, int sid, int64_t cap, int64_t *n_out, int32_t *cell, float *off, float *u,
                      float *w, int64_t *id)
{
    int r = check_ctx(c);
    if (r) return r;
    if (sid < 0 || sid >= c->nsp || !n_out) return fail(c, PIC_ERR_ARG, "bad species id");
    RecordView v;
    if ((r = record_view(c, sid, v))) return r;
    const Species &s = v.s;
    CK(cudaStreamSynchronize(c->stream));
    int cnt = 0;
    CK(cudaMemcpy(&cnt, s.count, sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<float4> P(cnt), Mo(cnt);
    std::vector<int> I(cnt);
    if (cnt > 0) {
        CK(cudaMemcpy(P.data(), s.pos, sizeof(float4) * cnt, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(Mo.data(), s.mom, sizeof(float4) * cnt, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(I.data(), s.id, sizeof(int) * cnt, cudaMemcpyDeviceToHost));
    }
    int64_t live = 0;
    for (int p = 0; p < cnt; p++) {
        int cb;
        std::memcpy(&cb, &P[p].w, sizeof(int));
        if (cb >= 0) live++;
    }
    *n_out = live;
    if (live > cap) return fail(c, PIC_ERR_CAPACITY, "output capacity below the live particle count");
    int64_t k = 0;
    for (int p = 0; p < cnt; p++) {
        int cb;
        std::memcpy(&cb, &P[p].w, sizeof(int));
        if (cb < 0) continue;
        if (cell) {
            cell[k] = c->cc.i(cb);
            cell[cap + k] = c->cc.j(cb);
            cell[2 * cap + k] = c->cc.k(cb);
        }
        if (off) {
            off[k] = P[p].x;
            off[cap + k] = P[p].y;
            off[2 * cap + k] = P[p].z;
        }
        if (u) {
            u[k] = Mo[p].x;
            u[cap + k] = Mo[p].y;
            u[2 * cap + k] = Mo[p].z;
        }
        if (w) w[k] = Mo[p].w;
        if (id) id[k] = I[p];
        k++;
    }
    return PIC_OK;
}

}  // extern "C"

namespace {

int moments_impl(pic_ctx *c, int sid, int run, int frame, double k_bunch, pic_moments *out)
{
    int r = check_ctx(c);
    if (r) return r;
    if (sid < 0 || sid >= c->nsp || !out) return fail(c, PIC_ERR_ARG, "bad species id");
    if (frame != PIC_FRAME_LAB && frame != PIC_FRAME_BOOSTED) return fail(c, PIC_ERR_ARG, "unknown frame");
    RecordView view;
    if ((r = record_view(c, sid, view))) return r;
    double v[20];
    CK(launch_moments(c, view.s, frame == PIC_FRAME_LAB ? PIC_FRAME_LAB : PIC_FRAME_BOOSTED, k_bunch, v, run));
    CK(launch_field_energy(c, &v[19], run));
    static_assert(sizeof(pic_moments) == 20 * sizeof(double), "pic_moments layout");
    std::memcpy(out, v, sizeof(v));
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_get_moments(pic_ctx *c, int sid, int frame, double k_bunch, pic_moments *out)
{
    return moments_impl(c, sid, -1, frame, k_bunch, out);
}

int pic_get_moments_run(pic_ctx *c, int sid, int run, int frame, double k_bunch, pic_moments *out)
{
    int r = check_ctx(c);
    if (r) return r;
    if (run < 0 || run >= c->runs) return fail(c, PIC_ERR_ARG, "run index outside the ensemble");
    return moments_impl(c, sid, run, frame, k_bunch, out);
}

int pic_get_time(pic_ctx *c, int64_t out[3])
{
    if (!c || !out) return PIC_ERR_ARG;
    out[0] = c->step;
    out[1] = c->shifts;
    out[2] = c->m_last;
    return PIC_OK;
}

int pic_get_count(pic_ctx *c, int sid, int64_t *n_out)
{
    int r = check_ctx(c);
    if (r) return r;
    if (sid < 0 || sid >= c->nsp || !n_out) return fail(c, PIC_ERR_ARG, "bad species id");
    RecordView v;
    if ((r = record_view(c, sid, v))) return r;
    CK(species_count_live(c, v.s, n_out));
    return PIC_OK;
}

int pic_trace_enable(pic_ctx *c, int on)
{
    int r = check_ctx(c);
    if (r) return r;
    c->trace_on = on != 0;
    return PIC_OK;
}

int pic_trace_read(pic_ctx *c, pic_trace *out)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!out) return fail(c, PIC_ERR_ARG, "trace output is NULL");
    CK(cudaStreamSynchronize(c->stream));
    for (auto &p : c->ev_pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.second.first, p.second.second));
        c->trace_ms[p.first] += ms;
        c->trace_n[p.first] += 1;
        c->ev_pool.push_back(p.second.first);
        c->ev_pool.push_back(p.second.second);
    }
    c->ev_pending.clear();
    for (int k = 0; k < 8; k++) {
        out->ms[k] = c->trace_ms[k];
        out->events[k] = c->trace_n[k];
        c->trace_ms[k] = 0;
        c->trace_n[k] = 0;
    }
    out->kernels = c->kernels;
    c->kernels = 0;
    unsigned long long nf = 0;
    CK(cudaMemcpyAsync(&nf, c->nfall, sizeof(nf), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemsetAsync(c->nfall, 0, sizeof(nf), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out->fallback = (int64_t)nf;
    return PIC_OK;
}

int pic_checkpoint(pic_ctx *c, int every_k)
{
    int r = check_ctx(c);
    if (r) return r;
    for (auto &st : c->ad_ckpt) free_state(c, st);
    for (auto &st : c->ad_rec) free_state(c, st);
    c->ad_ckpt.clear();
    c->ad_rec.clear();
    c->ad_rec_n = -1;
    c->ad_on = 0;
    if (every_k <= 0) return PIC_OK;
    if (c->order != 1) return fail(c, PIC_ERR_ARG, "the adjoint is built for the first-order shape");
    if (c->pusher != PIC_PUSHER_BORIS) return fail(c, PIC_ERR_ARG, "the adjoint reverses the Boris push");
    if (c->runs != 1 || c->moving || c->pml) return fail(c, PIC_ERR_ARG, "the adjoint needs one run, no window, no PML");
    for (int d = 0; d < 3; d++)
        if (c->bc[d][0] != PIC_BC_PERIODIC) return fail(c, PIC_ERR_ARG, "the adjoint needs a periodic grid");
    if (c->ext_type && std::isfinite(c->z_start) && c->ramp >= 0.0)
        return fail(c, PIC_ERR_ARG, "the adjoint needs an undulator without entrance ramp");
    if (c->ext_type == PIC_EXT_PLANAR_UNDULATOR_3D)
        return fail(c, PIC_ERR_ARG, "the adjoint is built for the 1-D planar undulator field");
    if (c->gather != PIC_GATHER_MOMENTUM)
        return fail(c, PIC_ERR_ARG, "the adjoint reverses the momentum-conserving gather");
    if (c->ion_G) return fail(c, PIC_ERR_ARG, "the adjoint does not differentiate the artificial ions");
    drop_graph(c);
    c->ad_on = 1;
    c->ad_every = every_k;
    c->ad_step0 = c->step;
    return PIC_OK;
}

int pic_backward(pic_ctx *c, const pic_adjoint_seed *seed, pic_grads *out)
{
    int r = check_ctx(c);
    if (r) return r;
    if (!seed || !out) return fail(c, PIC_ERR_ARG, "seed and out are required");
    if (!c->ad_on || c->ad_ckpt.empty()) return fail(c, PIC_ERR_STATE, "call pic_checkpoint before stepping");
    const int sid = seed->species_id;
    if (sid < 0 || sid >= c->nsp || c->sp[sid].lattice) return fail(c, PIC_ERR_ARG, "bad seed species");
    if (c->plasma && c->nprof > (int)(sizeof(out->dL_dprofile) / sizeof(double)))
        return fail(c, PIC_ERR_ARG, "profile has more nodes than pic_grads holds");
    CK(cudaStreamSynchronize(c->stream));
    const int64_t N = c->step, S0 = c->ad_step0, K = c->ad_every;
    std::memset(out, 0, sizeof(*out));
    // buffers
    const size_t f3 = 3 * (size_t)c->ncell;
    float *lE = nullptr, *lB = nullptr, *lJ = nullptr;
    double *lK = nullptr, *R = nullptr, *sums = nullptr, *grad = nullptr, *lw_plane = nullptr;
    std::vector<float4 *> lx(c->nsp, nullptr), lu(c->nsp, nullptr), lx2(c->nsp, nullptr), lu2(c->nsp, nullptr);
    std::vector<double *> lw(c->nsp, nullptr);
    int *inv = nullptr;
    int64_t max_ids = 1;
    for (int si = 0; si < c->nsp; si++) max_ids = std::max<int64_t>(max_ids, c->sp[si].next_id);
    StateSnap fin;   // the final state, restored at the end
    // every exit releases the scratch buffers and the saved final state (partial ones included)
    auto release = [&]() {
        free_state(c, fin);
        for (int si = 0; si < c->nsp; si++) {
            dfree(c, lx[si]);
            dfree(c, lu[si]);
            dfree(c, lx2[si]);
            dfree(c, lu2[si]);
            dfree(c, lw[si]);
        }
        dfree(c, lE);
        dfree(c, lB);
        dfree(c, lJ);
        dfree(c, lK);
        dfree(c, R);
        dfree(c, sums);
        dfree(c, grad);
        dfree(c, inv);
        dfree(c, lw_plane);
    };
    if ((r = alloc_zero(c, &lE, f3)) || (r = alloc_zero(c, &lB, f3)) || (r = alloc_zero(c, &lJ, f3)) ||
        (r = alloc_zero(c, &lK, 1)) || (r = alloc_zero(c, &R, (size_t)c->n[2])) || (r = alloc_zero(c, &sums, 3)) ||
        (r = alloc_zero(c, &grad, 64)) || (r = alloc_zero(c, &inv, (size_t)max_ids)) ||
        (c->plasma && (r = alloc_zero(c, &lw_plane, (size_t)c->sp[c->sp_i].plane_cap)))) {
        release();
        return r;
    }
    for (int si = 0; si < c->nsp; si++) {
        const Species &s = c->sp[si];
        if (s.lattice) continue;
        if ((r = alloc_zero(c, &lx[si], (size_t)s.cap)) || (r = alloc_zero(c, &lu[si], (size_t)s.cap)) ||
            (r = alloc_zero(c, &lx2[si], (size_t)s.cap)) || (r = alloc_zero(c, &lu2[si], (size_t)s.cap)) ||
            (r = alloc_zero(c, &lw[si], (size_t)std::max<int64_t>(s.next_id, 1)))) {
            release();
            return r;
        }
    }
    if ((r = save_state(c, fin, true))) {
        release();
        return r;
    }
    // records for one segment
    if ((int64_t)c->ad_rec.size() < K) c->ad_rec.resize((size_t)K);
    const int nseg = (int)((N - S0 + K - 1) / K);
    for (int j = nseg - 1; j >= 0 && r == PIC_OK; j--) {
        const int64_t s0 = S0 + (int64_t)j * K, e0 = std::min(N, s0 + K);
        if ((size_t)j >= c->ad_ckpt.size()) { r = fail(c, PIC_ERR_STATE, "missing adjoint checkpoint"); break; }
        if ((r = restore_state(c, c->ad_ckpt[(size_t)j]))) break;
        c->ad_rec_n = 0;
        for (int64_t n = s0; n < e0 && r == PIC_OK; n++) r = step_once(c);
        c->ad_rec_n = -1;
        if (r || (r = finish_records(c, (int)(e0 - s0)))) break;
        // The recomputed segment ends in the state the next checkpoint (or the final state) holds,
        // but the sort's order among particles is not reproducible: the adjoints carried over are
        // indexed in that checkpoint's order and are moved to the order the recomputed run has.
        const StateSnap &last = c->ad_rec[(size_t)(e0 - 1 - s0)];
        if (j == nseg - 1) {
            double h3[3] = {0, 0, 0};   // seed: the loss's gradient on the final positions
            const cudaError_t e = adj_bunch_seed(c, c->sp[sid], seed->k_bunch, sums, h3, lx[sid]);
            if (e != cudaSuccess) { r = fail_cuda(c, e, "adjoint seed"); break; }
            const double rr = std::sqrt(h3[0] * h3[0] + h3[1] * h3[1]);
            out->loss = h3[2] > 0 ? rr / h3[2] : 0.0;
        } else {
            const StateSnap &next = c->ad_ckpt[(size_t)j + 1];
            for (int si = 0; si < c->nsp && r == PIC_OK; si++) {
                if (c->sp[si].lattice) continue;
                const cudaError_t e = adj_remap(c, c->sp[si].id, last.sp[si].n, next.sp[si].id, next.sp[si].n, inv, lx[si],
                                                lu[si], lx2[si], lu2[si]);
                if (e != cudaSuccess) { r = fail_cuda(c, e, "adjoint remap"); break; }
                std::swap(lx[si], lx2[si]);
                std::swap(lu[si], lu2[si]);
            }
            if (r) break;
        }
        for (int64_t n = e0 - 1; n >= s0 && r == PIC_OK; n--) {
            const StateSnap &rec = c->ad_rec[(size_t)(n - s0)];
            if ((r = adj_fields(c, lE, lB, lJ) ? fail_cuda(c, cudaGetLastError(), "adjoint fields") : PIC_OK)) break;
            c->step = n;                 // the external field of step n
            ExtDev ext = ext_step(c);
            ext.clock = nullptr;
            for (int si = 0; si < c->nsp && r == PIC_OK; si++) {
                const Species &s = c->sp[si];
                if (s.lattice) {
                    const cudaError_t e = adj_ions(c, s, rec.sp[si].planes, lJ, R, lw_plane);
                    if (e != cudaSuccess) r = fail_cuda(c, e, "adjoint ions");
                    continue;
                }
                Species view = s;
                view.pos = rec.sp[si].pos;
                view.mom = rec.sp[si].mom;
                view.id = rec.sp[si].id;
                const cudaError_t e = adj_particles(c, view, rec.E, rec.B, lJ, lE, lB, lx[si], lu[si], lw[si], lK, ext,
                                                    rec.sp[si].n);
                if (e != cudaSuccess) r = fail_cuda(c, e, "adjoint particles");
            }
            if (r) break;
            if (rec.sorted) {
                // back to the order before the step's sort (the previous step's, or the checkpoint's)
                const StateSnap &before = n > s0 ? c->ad_rec[(size_t)(n - s0 - 1)] : c->ad_ckpt[(size_t)j];
                for (int si = 0; si < c->nsp && r == PIC_OK; si++) {
                    if (c->sp[si].lattice) continue;
                    // slots of particles the sort dropped (dummies) keep a zero adjoint
                    const cudaError_t e = adj_remap(c, before.sp[si].id, before.sp[si].n, rec.sp[si].id, rec.sp[si].n,
                                                    inv, lx[si], lu[si], lx2[si], lu2[si]);
                    if (e != cudaSuccess) { r = fail_cuda(c, e, "adjoint remap"); break; }
                    std::swap(lx[si], lx2[si]);
                    std::swap(lu[si], lu2[si]);
                }
            }
        }
    }
    c->step = N;
    if (r == PIC_OK && c->plasma) {
        const cudaError_t e = adj_profile_grad(c, lw[c->sp_e], c->sp[c->sp_e].next_id, lw_plane, grad);
        if (e != cudaSuccess) r = fail_cuda(c, e, "profile gradient");
    }
    if (r == PIC_OK) {
        double gk = 0.0, gp[64];
        cudaError_t e = cudaMemcpyAsync(&gk, lK, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gp, grad, sizeof(double) * 64, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            r = fail_cuda(c, e, "adjoint gradients");
        } else {
            out->dL_dK = gk;
            out->n_profile = c->plasma ? c->nprof : 0;
            for (int q = 0; q < out->n_profile; q++) out->dL_dprofile[q] = gp[q];
            r = restore_state(c, fin);
        }
    }
    release();
    return r;
}

int pic_destroy(pic_ctx *c)
{
    if (!c) return PIC_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (auto &p : c->ev_pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    while (!c->allocs.empty()) dfree(c, c->allocs.back().first);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return PIC_OK;
}

const char *pic_last_error(const pic_ctx *c)
{
    return c ? c->msg.c_str() : g_create_err.c_str();
}

}  // extern "C"

namespace gbpic {
// Message of a failed context-free call, reported by pic_last_error(NULL).
void set_global_error(const std::string &m) { g_create_err = m; }
}  // namespace gbpic

extern "C" {

}  // extern "C"
