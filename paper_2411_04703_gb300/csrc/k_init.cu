// FP64 kernels around the FP32 hot loop: the lab -> RRF transform of loaded particles
// (Eq. Lor1, Lor2, RRFVel; ballistic drift to t' = 0 as in Eq. BGauss/Belon), the injection
// of the lab-static plasma lattice entering the moving window (Eq. Nnormi, Vprime), the
// particle side of the window shift, and the FP64 beam moments in the RRF and back-
// transformed to the lab (inverse Eq. Lor1-Lor2, common lab time; spread bounded by Eq. DT).
#include "gbpic_internal.cuh"

#include <algorithm>
#include <cmath>

namespace gbpic {
namespace {

struct PlaceP {
    int n[3];
    int periodic[3];
    int mlo, mhi;
    int nzr;          // rows per run (ensembles)
    CellCode cc;
};

// Grid coordinate X of dimension d -> (cell, float offset); false outside the active region.
// A periodic z wraps inside the run whose first row is zb.
__device__ __forceinline__ bool place1(const PlaceP &g, int d, double X, float &o, int &c, int zb = 0)
{
    double fl = floor(X);
    float of = (float)(X - fl);
    if (of >= 1.f) { of = 0.f; fl += 1.0; }
    long long ci = (long long)fl;
    bool ok = true;
    const int per = d == 2 ? g.nzr : g.n[d];
    const int base = d == 2 ? zb : 0;
    if (g.periodic[d]) {
        ci = (ci - base) % per;
        if (ci < 0) ci += per;
        ci += base;
    } else if (ci < g.mlo || ci > g.n[d] - 1 - g.mhi) {
        ok = false;
        ci = 0;
    }
    c = (int)ci;
    o = of;
    return ok;
}

__device__ __forceinline__ bool place(const PlaceP &g, const double X[3], float o[3], int c[3], int zb = 0)
{
    const bool a = place1(g, 0, X[0], o[0], c[0]);
    const bool b = place1(g, 1, X[1], o[1], c[1]);
    const bool z = place1(g, 2, X[2], o[2], c[2], zb);
    return a && b && z;
}

struct LoadP {
    PlaceP g;
    double d[3], origin[3];
    double gR, bR, igR2;
    int frame, match;
    double qm, Aamp, ku, phase0;   // undulator vector potential A_x = Aamp sin(k_u z + phase0)
    int cosh_y;                    // 3-D field: A_x also carries cosh(k_u y), y from the axis ay
    double ay;
    long long n, stride;           // particles of this launch; component stride of x and u
    int id_base;
    int zb;                        // first row of the run the particles are loaded into
};

__global__ void k_load(SpeciesDev sp, LoadP p, const double *x, const double *u, const double *w, int *err)
{
    const long long n = p.n;
    const int base = sp.count[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long st = p.stride;
        double xi[3] = {x[i], x[st + i], x[2 * st + i]};
        double ui[3] = {u[i], u[st + i], u[2 * st + i]};
        const double wi = w ? w[i] : 1.0;
        if (p.frame == PIC_FRAME_LAB && p.match) {
            // matched entry: lab energy kept, transverse canonical momentum u_x + (q/m) A_x = 0
            const double g = sqrt(1.0 + ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]);
            const double zlab = xi[2] + p.gR * p.origin[2] * p.d[2];
            const double ch = p.cosh_y ? cosh(p.ku * (xi[1] + p.origin[1] * p.d[1] - p.ay)) : 1.0;
            ui[0] += -p.qm * p.Aamp * ch * sin(p.ku * zlab + p.phase0);
            ui[2] = sqrt(g * g - 1.0 - ui[0] * ui[0] - ui[1] * ui[1]);
        }
        double xp[3], up[3];
        if (p.frame == PIC_FRAME_LAB) {
            const double up2 = ui[0] * ui[0] + ui[1] * ui[1];
            const double g = sqrt(1.0 + up2 + ui[2] * ui[2]);
            double uzp, gp;
            if (ui[2] >= 0.0) {
                // u_z - beta_R g and g - beta_R u_z without cancellation
                uzp = p.gR * ((g * g * p.igR2 - 1.0 - up2) / (ui[2] + p.bR * g));
                gp = p.gR * ((1.0 + up2 + ui[2] * ui[2] * p.igR2) / (g + p.bR * ui[2]));
            } else {
                uzp = p.gR * (ui[2] - p.bR * g);
                gp = p.gR * (g - p.bR * ui[2]);
            }
            // event (x, t = 0) -> (x', t' = -gamma_R beta_R z); drift to t' = 0
            const double dtp = p.gR * p.bR * xi[2];
            up[0] = ui[0];
            up[1] = ui[1];
            up[2] = uzp;
            xp[0] = xi[0] + dtp * up[0] / gp;
            xp[1] = xi[1] + dtp * up[1] / gp;
            xp[2] = p.gR * xi[2] + dtp * up[2] / gp;
        } else {
            for (int d = 0; d < 3; d++) { xp[d] = xi[d]; up[d] = ui[d]; }
        }
        double X[3];
        for (int d = 0; d < 3; d++) X[d] = xp[d] / p.d[d] + p.origin[d];
        X[2] += p.zb;
        float o[3];
        int c[3];
        const bool ok = place(p.g, X, o, c, p.zb);
        const long long slot = (long long)base + i;
        if (slot >= sp.cap) { atomicOr(err, ERR_CAPACITY); continue; }
        sp.pos[slot] = make_float4(o[0], o[1], o[2], __int_as_float(ok ? p.g.cc.pack(c[0], c[1], c[2]) : -1));
        sp.mom[slot] = make_float4((float)up[0], (float)up[1], (float)up[2], (float)wi);
        sp.id[slot] = p.id_base + (int)i;
    }
}

__global__ void k_bump(int *count, long long add, int cap, int *err)
{
    long long v = (long long)count[0] + add;
    if (v > cap) { atomicOr(err, ERR_CAPACITY); v = cap; }
    count[0] = (int)v;
}

struct InjP {
    PlaceP g;
    long long m0, count;
    int per_plane, nxr, x0, y0, ppc[3];
    double zshift;       // beta_R t' / dz + window shifts (cells)
    double gR, dz, wfac;
    float uz;
    const double *prof;  // [2][nprof]: z nodes then densities
    int nprof;
    int id_e, id_i;
    PlaneRec *planes;    // ions as a lattice species: plane m goes to slot m mod plane_cap
    long long plane_cap;
    const double *run_scale;  // ensembles: density scale of each run (plane m belongs to the run
                              // holding its unshifted row); NULL: one run
};

__device__ double profile(const double *prof, int np, double z)
{
    if (np <= 0 || z < prof[0] || z > prof[np - 1]) return 0.0;
    for (int i = 0; i + 1 < np; i++) {
        if (z <= prof[i + 1]) {
            const double h = prof[i + 1] - prof[i];
            const double r = h > 0.0 ? (z - prof[i]) / h : 0.0;
            return prof[np + i] + r * (prof[np + i + 1] - prof[np + i]);
        }
    }
    return prof[2 * np - 1];
}

// Lattice point t of planes m0.. (transverse index r = t mod per_plane, ppc_x fastest, then
// ppc_y, then the cells of the x range, then y): grid coordinates of the point.
__device__ __forceinline__ void lattice_point(const InjP &p, long long t, long long &m, int &r, double X[3])
{
    m = p.m0 + t / p.per_plane;
    r = (int)(t % p.per_plane);
    int q = r;
    const int a = q % p.ppc[0];
    q /= p.ppc[0];
    const int b = q % p.ppc[1];
    q /= p.ppc[1];
    const int ii = q % p.nxr, jj = q / p.nxr;
    X[0] = p.x0 + ii + (a + 0.5) / p.ppc[0];
    X[1] = p.y0 + jj + (b + 0.5) / p.ppc[1];
    X[2] = ((double)m + 0.5) / p.ppc[2] - p.zshift;
}

__global__ void k_inject(SpeciesDev se, SpeciesDev si, InjP p, int *err)
{
    const int base_e = se.count[0], base_i = p.planes ? 0 : si.count[0];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < p.count; t += (long long)gridDim.x * blockDim.x) {
        long long m;
        int r;
        double X[3];
        lattice_point(p, t, m, r, X);
        double zc = ((double)m + 0.5) / p.ppc[2];
        int zb = 0;
        double scale = 1.0;
        if (p.run_scale) {
            const int run = (int)floor(zc / p.g.nzr);
            zb = run * p.g.nzr;
            zc -= zb;   // the profile is given in each run's own coordinates
            scale = p.run_scale[run];
        }
        const double dens = p.gR * profile(p.prof, p.nprof, p.gR * zc * p.dz) * scale;
        float o[3];
        int c[3];
        const bool ok = place(p.g, X, o, c, zb) && dens > 0.0;
        const float4 P = make_float4(o[0], o[1], o[2], __int_as_float(ok ? p.g.cc.pack(c[0], c[1], c[2]) : -1));
        const float4 Mo = make_float4(0.f, 0.f, p.uz, (float)(dens * p.wfac));
        const long long se_slot = base_e + t;
        if (se_slot >= se.cap) { atomicOr(err, ERR_CAPACITY); continue; }
        se.pos[se_slot] = P;
        se.mom[se_slot] = Mo;
        se.id[se_slot] = p.id_e + (int)t;
        if (p.planes) {
            if (r != 0) continue;
            // one plane record: the z placement, the weight and the plane's first id
            PlaneRec &slot = p.planes[m % p.plane_cap];
            if (slot.kz >= 0) { atomicOr(err, ERR_CAPACITY); continue; }
            float oz;
            int kz;
            const bool okz = place1(p.g, 2, X[2], oz, kz, zb) && dens > 0.0;
            slot = PlaneRec{oz, okz ? kz : -1, Mo.w, p.id_i + (int)t};
            continue;
        }
        const long long si_slot = base_i + t;
        if (si_slot >= si.cap) { atomicOr(err, ERR_CAPACITY); continue; }
        si.pos[si_slot] = P;
        si.mom[si_slot] = Mo;
        si.id[si_slot] = p.id_i + (int)t;
    }
}

// Transverse profile of the lattice species: T(i) = sum over the lattice's points x along dim
// d (cells lo .. hi-1, ppc points each, placed as at injection) of S(i - x); periodic dims wrap.
__global__ void k_lattice_profile(PlaceP g, int d, int lo, int hi, int ppc, int order, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n[d]) return;
    double acc = 0.0;
    for (int cell = lo; cell < hi; cell++)
        for (int a = 0; a < ppc; a++) {
            float o;
            int ci;
            if (!place1(g, d, cell + (a + 0.5) / ppc, o, ci)) continue;
            double x = (double)i - ((double)ci + (double)o);
            if (!g.periodic[d]) {
                acc += shape_weight(order, x);
                continue;
            }
            // every periodic image within the shape's reach (more than one when the dim has
            // fewer cells than the stencil, e.g. n = 1 in a 2-D geometry)
            x -= g.n[d] * rint(x / g.n[d]);
            for (int m = -2; m <= 2; m++) acc += shape_weight(order, x + (double)m * g.n[d]);
        }
    out[i] = (float)acc;
}

// Particle records of the lattice species, materialised from its planes: slot s of the plane
// ring and transverse index r give record s * per_plane + r (dropped planes give dummies).
__global__ void k_lattice_records(SpeciesDev out, const PlaneRec *planes, long long cap, InjP p)
{
    const long long n = cap * p.per_plane;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out.count[0] = (int)n;
        out.count[1] = 0;
        out.count[2] = 0;
    }
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const PlaneRec pl = planes[t / p.per_plane];
        long long m;
        int r;
        double X[3];
        lattice_point(p, t, m, r, X);
        float ox, oy;
        int cx, cy;
        const bool okx = place1(p.g, 0, X[0], ox, cx);
        const bool oky = place1(p.g, 1, X[1], oy, cy);
        const bool ok = pl.kz >= 0 && okx && oky;
        out.pos[t] = make_float4(ox, oy, pl.oz, __int_as_float(ok ? p.g.cc.pack(cx, cy, pl.kz) : -1));
        out.mom[t] = make_float4(0.f, 0.f, p.uz, pl.w);
        out.id[t] = pl.id0 + r;
    }
}

__global__ void k_shift_particles(SpeciesDev sp, int mlo, CellCode cc)
{
    const int n = sp.count[0];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int cell = __float_as_int(sp.pos[p].w);
        if (cell < 0) continue;
        const int k = cc.k(cell) - 1;
        sp.pos[p].w = __int_as_float(k < mlo ? -1 : cc.pack(cc.i(cell), cc.j(cell), k));
    }
}

// ------------------------------------------------------------------ FP64 moments
struct MomP {
    double d[3];
    double shifts, tp, gR, bR, igR2, mass, k;
    int frame, pass;
    double mean_t;
    double mean[7];   // x y z ux uy uz gamma
    CellCode cc;
    int k_lo, k_hi;   // rows of the run whose particles are summed (ensembles; whole grid otherwise)
};

constexpr int kMomK = 10;

__device__ __forceinline__ void particle_frame(const MomP &p, float4 P, float4 Mo, double x[3], double u[3],
                                               double &g, double &t)
{
    const int cell = __float_as_int(P.w);
    x[0] = ((double)p.cc.i(cell) + (double)P.x) * p.d[0];
    x[1] = ((double)p.cc.j(cell) + (double)P.y) * p.d[1];
    x[2] = ((double)(p.cc.k(cell) - p.k_lo) + (double)P.z + p.shifts) * p.d[2];
    u[0] = Mo.x; u[1] = Mo.y; u[2] = Mo.z;
    const double up2 = u[0] * u[0] + u[1] * u[1];
    const double gp = sqrt(1.0 + up2 + u[2] * u[2]);
    t = p.tp;
    g = gp;
    if (p.frame == PIC_FRAME_LAB) {
        const double zp = x[2];
        x[2] = p.gR * (zp + p.bR * p.tp);
        t = p.gR * (p.tp + p.bR * zp);
        double uz, gl;
        if (u[2] >= 0.0) {
            uz = p.gR * (u[2] + p.bR * gp);
            gl = p.gR * (gp + p.bR * u[2]);
        } else {
            uz = p.gR * ((u[2] * u[2] * p.igR2 - p.bR * p.bR * (1.0 + up2)) / (u[2] - p.bR * gp));
            gl = p.gR * ((1.0 + up2 + u[2] * u[2] * p.igR2) / (gp - p.bR * u[2]));
        }
        u[2] = uz;
        g = gl;
    }
}

__global__ void k_moments(SpeciesDev sp, MomP p, double *partial)
{
    double acc[kMomK];
#pragma unroll
    for (int j = 0; j < kMomK; j++) acc[j] = 0.0;
    const int n = sp.count[0];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const float4 P = sp.pos[q];
        if (__float_as_int(P.w) < 0) continue;
        const int kc = p.cc.k(__float_as_int(P.w));
        if (kc < p.k_lo || kc >= p.k_hi) continue;
        const float4 Mo = sp.mom[q];
        const double w = Mo.w;
        double x[3], u[3], g, t;
        particle_frame(p, P, Mo, x, u, g, t);
        if (p.pass == 0) {
            acc[0] += w;
            acc[1] += w * t;
            acc[2] += 1.0;
            continue;
        }
        if (p.frame == PIC_FRAME_LAB) {
            const double dl = p.mean_t - t;
            for (int d = 0; d < 3; d++) x[d] += dl * u[d] / g;
        }
        if (p.pass == 1) {
            acc[0] += w * x[0]; acc[1] += w * x[1]; acc[2] += w * x[2];
            acc[3] += w * u[0]; acc[4] += w * u[1]; acc[5] += w * u[2];
            acc[6] += w * g;
            acc[7] += w * p.mass * (g - 1.0);
        } else {
            const double dx = x[0] - p.mean[0], dy = x[1] - p.mean[1], dz = x[2] - p.mean[2];
            const double dux = u[0] - p.mean[3], duy = u[1] - p.mean[4], dg = g - p.mean[6];
            acc[0] += w * dx * dx; acc[1] += w * dy * dy; acc[2] += w * dz * dz;
            acc[3] += w * dux * dux; acc[4] += w * duy * duy;
            acc[5] += w * dx * dux; acc[6] += w * dy * duy;
            acc[7] += w * dg * dg;
            double sn, cs;
            sincos(p.k * dz, &sn, &cs);
            acc[8] += w * cs;
            acc[9] -= w * sn;
        }
    }
    __shared__ double ws[kMomK][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMomK; j++) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) ws[j][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kMomK) {
        double v = 0.0;
        for (int k2 = 0; k2 < (int)(blockDim.x >> 5); k2++) v += ws[threadIdx.x][k2];
        partial[blockIdx.x * kMomK + threadIdx.x] = v;
    }
}

__global__ void k_wmax(SpeciesDev sp, double *partial)
{
    double m = 0.0;
    const int n = sp.count[0];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        m = fmax(m, fabs((double)sp.mom[p].w));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) m = fmax(m, ws[k]);
        partial[blockIdx.x] = m;
    }
}

__global__ void k_absmax_f64(const double *a, long long n, double *partial)
{
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(a[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) m = fmax(m, ws[k]);
        partial[blockIdx.x] = m;
    }
}

__global__ void k_count_live(SpeciesDev sp, unsigned long long *out)
{
    unsigned long long cnt = 0;
    const int n = sp.count[0];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        cnt += __float_as_int(sp.pos[p].w) >= 0;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

PlaceP place_params(const pic_ctx *c)
{
    PlaceP g;
    for (int d = 0; d < 3; d++) {
        g.n[d] = c->n[d];
        g.periodic[d] = c->bc[d][0] == PIC_BC_PERIODIC;
    }
    g.mlo = c->order == 1 ? 1 : 2;
    g.mhi = c->order == 1 ? 2 : 3;
    g.nzr = c->nzr;
    g.cc = c->cc;
    return g;
}

}  // namespace

// Loads n particles into run `run` (0 for a single run); dx, du: device [3][stride] arrays
// (component stride `stride`), dw: device [n] or NULL.
cudaError_t launch_load(pic_ctx *c, int si, int64_t n, const double *dx, const double *du, const double *dw,
                        int frame, const double origin[3], int match, int64_t id_base, int run, int64_t stride)
{
    Species &s = c->sp[si];
    LoadP p;
    p.g = place_params(c);
    for (int d = 0; d < 3; d++) { p.d[d] = c->d[d]; p.origin[d] = origin[d]; }
    p.gR = c->gR;
    p.bR = c->bR;
    p.igR2 = 1.0 / (c->gR * c->gR);
    p.frame = frame;
    p.match = match && (c->ext_type == PIC_EXT_PLANAR_UNDULATOR || c->ext_type == PIC_EXT_PLANAR_UNDULATOR_3D);
    p.cosh_y = c->ext_type == PIC_EXT_PLANAR_UNDULATOR_3D;
    p.ay = 0.5 * c->n[1] * c->d[1];
    p.qm = s.q / s.m;
    const double B0 = c->B0_run.empty() ? c->B0 : c->B0_run[run];
    p.Aamp = c->ku > 0 ? B0 / c->ku : 0.0;
    p.ku = c->ku;
    p.phase0 = c->phase0;
    p.n = n;
    p.stride = stride;
    p.id_base = (int)id_base;
    p.zb = run * c->nzr;
    if (n > 0) {
        k_load<<<c->num_sms * 4, 256, 0, c->stream>>>(species_dev(c, s), p, dx, du, dw, c->err);
        c->kernels++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_bump<<<1, 1, 0, c->stream>>>(s.count, n, (int)s.cap, c->err);
    c->kernels++;
    return cudaGetLastError();
}

cudaError_t launch_inject(pic_ctx *c, int64_t m0, int64_t m1)
{
    if (m1 < m0) return cudaSuccess;
    Species &se = c->sp[c->sp_e], &si = c->sp[c->sp_i];
    InjP p;
    p.g = place_params(c);
    p.nxr = c->xr[1] - c->xr[0];
    const int nyr = c->xr[3] - c->xr[2];
    p.x0 = c->xr[0];
    p.y0 = c->xr[2];
    for (int d = 0; d < 3; d++) p.ppc[d] = c->ppc[d];
    p.per_plane = p.nxr * nyr * c->ppc[0] * c->ppc[1];
    p.m0 = m0;
    p.count = (m1 - m0 + 1) * (int64_t)p.per_plane;
    p.zshift = c->bR * (double)c->step * c->dt / c->d[2] + (double)c->shifts;
    p.gR = c->gR;
    p.dz = c->d[2];
    p.wfac = c->d[0] * c->d[1] * c->d[2] / ((double)c->ppc[0] * c->ppc[1] * c->ppc[2]);
    p.uz = (float)(-sqrt(c->gR * c->gR - 1.0));
    p.prof = c->prof;
    p.nprof = c->nprof;
    p.id_e = (int)se.next_id;
    p.id_i = (int)si.next_id;
    p.planes = si.lattice ? si.planes : nullptr;
    p.plane_cap = si.plane_cap;
    p.run_scale = c->runs > 1 ? c->dens_scale : nullptr;
    if (p.count <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((p.count + 255) / 256, (long long)c->num_sms * 16);
    k_inject<<<(unsigned)blocks, 256, 0, c->stream>>>(species_dev(c, se), species_dev(c, si), p, c->err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bump<<<1, 1, 0, c->stream>>>(se.count, p.count, (int)se.cap, c->err);
    c->kernels += 2;
    if (!si.lattice) {
        k_bump<<<1, 1, 0, c->stream>>>(si.count, p.count, (int)si.cap, c->err);
        c->kernels++;
        si.bound += p.count;
    }
    se.next_id += p.count;
    si.next_id += p.count;
    se.bound += p.count;
    return cudaGetLastError();
}

namespace {
InjP lattice_params(pic_ctx *c)
{
    InjP p{};
    p.g = place_params(c);
    p.nxr = c->xr[1] - c->xr[0];
    p.x0 = c->xr[0];
    p.y0 = c->xr[2];
    for (int d = 0; d < 3; d++) p.ppc[d] = c->ppc[d];
    p.per_plane = p.nxr * (c->xr[3] - c->xr[2]) * c->ppc[0] * c->ppc[1];
    p.uz = (float)(-sqrt(c->gR * c->gR - 1.0));
    return p;
}
}  // namespace

cudaError_t launch_lattice_profiles(pic_ctx *c, int si)
{
    const Species &s = c->sp[si];
    const PlaceP g = place_params(c);
    k_lattice_profile<<<(c->n[0] + 127) / 128, 128, 0, c->stream>>>(g, 0, c->xr[0], c->xr[1], c->ppc[0], c->order, s.tx);
    k_lattice_profile<<<(c->n[1] + 127) / 128, 128, 0, c->stream>>>(g, 1, c->xr[2], c->xr[3], c->ppc[1], c->order, s.ty);
    c->kernels += 2;
    return cudaGetLastError();
}

// out: pos, mom, id of plane_cap * per_plane slots and count[4], allocated by the caller.
cudaError_t launch_lattice_records(pic_ctx *c, int si, Species &out)
{
    const Species &s = c->sp[si];
    const InjP p = lattice_params(c);
    const long long n = s.plane_cap * p.per_plane;
    const long long blocks = std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)c->num_sms * 16));
    k_lattice_records<<<(unsigned)blocks, 256, 0, c->stream>>>(species_dev(c, out), s.planes, s.plane_cap, p);
    c->kernels++;
    return cudaGetLastError();
}

cudaError_t species_wmax(pic_ctx *c, int si, double *out)
{
    const int blocks = 256;
    k_wmax<<<blocks, 256, 0, c->stream>>>(species_dev(c, c->sp[si]), c->red);
    c->kernels++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::vector<double> part(blocks);
    e = cudaMemcpyAsync(part.data(), c->red, blocks * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    double m = 0.0;
    for (double v : part) m = std::max(m, v);
    *out = m;
    return cudaSuccess;
}

// Largest |a[i]| of a device FP64 array (synchronous).
cudaError_t absmax_f64(pic_ctx *c, const double *a, int64_t n, double *out)
{
    const int blocks = 256;
    k_absmax_f64<<<blocks, 256, 0, c->stream>>>(a, n, c->red);
    c->kernels++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::vector<double> part(blocks);
    e = cudaMemcpyAsync(part.data(), c->red, sizeof(double) * blocks, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    double m = 0.0;
    for (double v : part) m = std::max(m, v);
    *out = m;
    return cudaSuccess;
}

cudaError_t species_count_live(pic_ctx *c, const Species &s, int64_t *out)
{
    unsigned long long *d = reinterpret_cast<unsigned long long *>(c->red);
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    k_count_live<<<c->num_sms * 4, 256, 0, c->stream>>>(species_dev(c, s), d);
    c->kernels++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned long long h = 0;
    if ((e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    *out = (int64_t)h;
    return cudaSuccess;
}

cudaError_t launch_shift_particles(pic_ctx *c, int si)
{
    k_shift_particles<<<c->num_sms * 8, 256, 0, c->stream>>>(species_dev(c, c->sp[si]), c->order == 1 ? 1 : 2, c->cc);
    c->kernels++;
    return cudaGetLastError();
}

// FP64 moments of species s, over the whole grid (run < 0) or over one run of an ensemble (its
// positions then in the run's own coordinates).
cudaError_t launch_moments(pic_ctx *c, const Species &s, int frame, double k, double *out, int run)
{
    MomP p{};
    p.cc = c->cc;
    p.k_lo = run < 0 ? 0 : run * c->nzr;
    p.k_hi = run < 0 ? c->n[2] : (run + 1) * c->nzr;
    for (int d = 0; d < 3; d++) p.d[d] = c->d[d];
    p.shifts = (double)c->shifts;
    p.tp = (double)c->step * c->dt;
    p.gR = c->gR;
    p.bR = c->bR;
    p.igR2 = 1.0 / (c->gR * c->gR);
    p.mass = s.m;
    p.k = k;
    p.frame = frame;
    const int blocks = 512;
    std::vector<double> part((size_t)blocks * kMomK);
    double sums[3][kMomK];
    for (int pass = 0; pass < 3; pass++) {
        p.pass = pass;
        k_moments<<<blocks, 256, 0, c->stream>>>(species_dev(c, s), p, c->red);
        c->kernels++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(part.data(), c->red, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return e;
        for (int j = 0; j < kMomK; j++) {
            double v = 0.0;
            for (int b = 0; b < blocks; b++) v += part[(size_t)b * kMomK + j];
            sums[pass][j] = v;
        }
        const double sw = sums[0][0];
        if (pass == 0) {
            p.mean_t = sw > 0 ? sums[0][1] / sw : p.tp;
        } else if (pass == 1) {
            for (int j = 0; j < 7; j++) p.mean[j] = sw > 0 ? sums[1][j] / sw : 0.0;
        }
    }
    const double sw = sums[0][0];
    for (int j = 0; j < 20; j++) out[j] = 0.0;
    out[0] = sums[0][2];
    out[1] = sw;
    out[2] = s.q * sw;
    if (sw > 0) {
        const double *cs = sums[2];
        for (int d = 0; d < 3; d++) {
            out[3 + d] = p.mean[d];
            out[6 + d] = sqrt(cs[d] / sw);
            out[9 + d] = p.mean[3 + d];
        }
        out[12] = p.mean[6];
        out[13] = sqrt(cs[7] / sw) / p.mean[6];
        const double ex = (cs[0] / sw) * (cs[3] / sw) - (cs[5] / sw) * (cs[5] / sw);
        const double ey = (cs[1] / sw) * (cs[4] / sw) - (cs[6] / sw) * (cs[6] / sw);
        out[14] = sqrt(ex > 0 ? ex : 0.0);
        out[15] = sqrt(ey > 0 ? ey : 0.0);
        out[16] = sqrt(cs[8] * cs[8] + cs[9] * cs[9]) / sw;
        out[17] = sums[1][7];
        out[18] = p.mean_t;
    }
    return cudaSuccess;
}

}  // namespace gbpic
