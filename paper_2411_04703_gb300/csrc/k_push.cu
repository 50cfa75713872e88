// Fused particle kernel of one boosted-frame PIC step (sm_103a).
//
// Per particle: gather E^n, B^n with the particle shape at each component's Yee point, add
// the analytic external undulator field of the RRF (Eq. M1-M4 applied to the lab field at
// lab z = gamma_R (z' + beta_R t'), Eq. Vprime), leap-frog (Boris) push u^{n-1/2} -> u^{n+1/2},
// move x^n -> x^{n+1} (integer cell + FP32 offset), and the Esirkepov charge-conserving current
// J^{n+1/2} (Eq. Max3-Max4 solved by current weighting).
//
// Work decomposition: particles are sorted by tile; a persistent grid pulls (tile, chunk)
// work items from an atomic counter.  For a tile item the CTA stages the E/B region of the
// tile (+ drift margin + stencil halo) in shared memory, accumulates the current of its
// particles in a shared-memory J region with shared atomics, and flushes the region to the
// global J once with global atomics.  Particles that drifted beyond the margin since the last
// sort, and appended (unsorted) particles, take the global-memory path.
#include "gbpic_internal.cuh"

namespace gbpic {
namespace {

// ------------------------------------------------------------------ shape weights
template <int ORDER> struct Shape;

template <> struct Shape<1> {
    static constexpr int N = 2;   // gather nodes per dim
    static constexpr int L = 3;   // Esirkepov window per dim
    // nodes at integer positions: start c + s
    __device__ __forceinline__ static void unst(float o, int &s, float w[2]) {
        s = 0; w[0] = 1.f - o; w[1] = o;
    }
    // nodes at positions m + 1/2
    __device__ __forceinline__ static void stag(float o, int &s, float w[2]) {
        const bool hi = o >= 0.5f;
        const float f = hi ? o - 0.5f : o + 0.5f;
        s = hi ? 0 : -1; w[0] = 1.f - f; w[1] = f;
    }
    // S0, S1 on the window [c + st, c + st + L) for a move from (c, o) to (c + s, o1)
    __device__ __forceinline__ static void window(float o, int s, float o1, int &st, float S0[3], float S1[3]) {
        const int mn = min(s, 0);
        st = mn;
        const int i0 = -mn, i1 = s - mn;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            S0[a] = (a == i0) ? 1.f - o : ((a == i0 + 1) ? o : 0.f);
            S1[a] = (a == i1) ? 1.f - o1 : ((a == i1 + 1) ? o1 : 0.f);
        }
    }
};

template <> struct Shape<2> {
    static constexpr int N = 3;
    static constexpr int L = 4;
    __device__ __forceinline__ static void tsc(float dl, float w[3]) {
        const float a = 0.5f - dl, b = 0.5f + dl;
        w[0] = 0.5f * a * a; w[1] = 0.75f - dl * dl; w[2] = 0.5f * b * b;
    }
    __device__ __forceinline__ static void unst(float o, int &s, float w[3]) {
        const int b = o >= 0.5f;
        s = b - 1; tsc(o - (float)b, w);
    }
    __device__ __forceinline__ static void stag(float o, int &s, float w[3]) {
        s = -1; tsc(o - 0.5f, w);
    }
    __device__ __forceinline__ static void window(float o, int s, float o1, int &st, float S0[4], float S1[4]) {
        const int b0 = o >= 0.5f, b1r = o1 >= 0.5f;
        const int sb = s + b1r - b0;           // shift of the nearest node, -1..1
        const int mn = min(sb, 0);
        st = b0 - 1 + mn;
        const int i0 = -mn, i1 = sb - mn;
        float w0[3], w1[3];
        tsc(o - (float)b0, w0);
        tsc(o1 - (float)b1r, w1);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int k0 = a - i0, k1 = a - i1;
            S0[a] = k0 == 0 ? w0[0] : (k0 == 1 ? w0[1] : (k0 == 2 ? w0[2] : 0.f));
            S1[a] = k1 == 0 ? w1[0] : (k1 == 1 ? w1[1] : (k1 == 2 ? w1[2] : 0.f));
        }
    }
};

// ------------------------------------------------------------------ field / current access
// Shared-memory region of a tile: node (c + x) of the particle's cell c sits at local
// coordinate l + x.
struct SmemAcc {
    const float *sF;
    float *sJ;
    int Rx, R2, R3;
    int base;   // local linear index of the particle's cell
    __device__ __forceinline__ float f(int comp, int x, int y, int z) const {
        return sF[comp * R3 + base + z * R2 + y * Rx + x];
    }
    __device__ __forceinline__ void j(int comp, int x, int y, int z, float v) const {
        atomicAdd(&sJ[comp * R3 + base + z * R2 + y * Rx + x], v);
    }
};

// Global-memory access with periodic wrap; outside a non-periodic face fields read as 0 and a
// current contribution raises ERR_INDEX (particle margins make this unreachable).
struct GlobAcc {
    const float *E, *B;
    float *J;
    GridDev g;
    int c[3];
    int *err;
    __device__ __forceinline__ long long node(int x, int y, int z) const {
        int p[3] = {c[0] + x, c[1] + y, c[2] + z};
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (p[d] < 0 || p[d] >= g.n[d]) {
                if (!g.periodic[d]) return -1;
                p[d] = p[d] < 0 ? p[d] + g.n[d] : p[d] - g.n[d];
            }
        }
        return ((long long)p[2] * g.n[1] + p[1]) * g.n[0] + p[0];
    }
    __device__ __forceinline__ float f(int comp, int x, int y, int z) const {
        const long long ix = node(x, y, z);
        if (ix < 0) return 0.f;
        const float *F = comp < 3 ? E + comp * g.ncell : B + (comp - 3) * g.ncell;
        return __ldg(F + ix);
    }
    __device__ __forceinline__ void j(int comp, int x, int y, int z, float v) const {
        const long long ix = node(x, y, z);
        if (ix < 0) { atomicOr(err, ERR_INDEX); return; }
        atomicAdd(&J[comp * g.ncell + ix], v);
    }
};

template <int N, class Acc>
__device__ __forceinline__ float gather(const Acc &a, int comp, int sx, int sy, int sz,
                                        const float *wx, const float *wy, const float *wz)
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < N; k++) {
        float sk = 0.f;
#pragma unroll
        for (int j = 0; j < N; j++) {
            float sj = 0.f;
#pragma unroll
            for (int i = 0; i < N; i++) sj = fmaf(wx[i], a.f(comp, sx + i, sy + j, sz + k), sj);
            sk = fmaf(wy[j], sj, sk);
        }
        s = fmaf(wz[k], sk, s);
    }
    return s;
}

// Esirkepov current of one particle: W_c = DS_c (S0_a S0_b + DS_a S0_b/2 + S0_a DS_b/2 +
// DS_a DS_b/3) for the two other dims a, b, prefix-summed along c from the window start.
template <int L, class Acc>
__device__ __forceinline__ void esirkepov(const Acc &acc, const int st[3], const float S0[3][L],
                                          const float DS[3][L], const float fac[3])
{
    // J_x
#pragma unroll
    for (int k = 0; k < L; k++)
#pragma unroll
        for (int j = 0; j < L; j++) {
            const float Y = S0[1][j] * S0[2][k] + 0.5f * DS[1][j] * S0[2][k] + 0.5f * S0[1][j] * DS[2][k] +
                            (1.f / 3.f) * DS[1][j] * DS[2][k];
            float run = 0.f;
#pragma unroll
            for (int i = 0; i < L - 1; i++) {
                run = fmaf(DS[0][i], Y, run);
                if (run != 0.f) acc.j(0, st[0] + i, st[1] + j, st[2] + k, fac[0] * run);
            }
        }
    // J_y
#pragma unroll
    for (int k = 0; k < L; k++)
#pragma unroll
        for (int i = 0; i < L; i++) {
            const float Y = S0[2][k] * S0[0][i] + 0.5f * DS[2][k] * S0[0][i] + 0.5f * S0[2][k] * DS[0][i] +
                            (1.f / 3.f) * DS[2][k] * DS[0][i];
            float run = 0.f;
#pragma unroll
            for (int j = 0; j < L - 1; j++) {
                run = fmaf(DS[1][j], Y, run);
                if (run != 0.f) acc.j(1, st[0] + i, st[1] + j, st[2] + k, fac[1] * run);
            }
        }
    // J_z
#pragma unroll
    for (int j = 0; j < L; j++)
#pragma unroll
        for (int i = 0; i < L; i++) {
            const float Y = S0[0][i] * S0[1][j] + 0.5f * DS[0][i] * S0[1][j] + 0.5f * S0[0][i] * DS[1][j] +
                            (1.f / 3.f) * DS[0][i] * DS[1][j];
            float run = 0.f;
#pragma unroll
            for (int k = 0; k < L - 1; k++) {
                run = fmaf(DS[2][k], Y, run);
                if (run != 0.f) acc.j(2, st[0] + i, st[1] + j, st[2] + k, fac[2] * run);
            }
        }
}

// One particle through the whole step.  Returns false when the particle left the domain
// through a non-periodic face (it becomes a dummy particle and deposits nothing).
template <int ORDER, bool FROZEN, class Acc>
__device__ __forceinline__ bool advance(const Acc &acc, float o[3], int c[3], float4 &mo,
                                        const SpeciesDev &sp, const GridDev &g, const ExtDev &ext,
                                        int *err)
{
    using S = Shape<ORDER>;
    constexpr int N = S::N, L = S::L;
    float u[3] = {mo.x, mo.y, mo.z};
    if (!FROZEN) {
        int su[3], ss[3];
        float wu[3][N], ws[3][N];
#pragma unroll
        for (int d = 0; d < 3; d++) { S::unst(o[d], su[d], wu[d]); S::stag(o[d], ss[d], ws[d]); }
        float E[3], B[3];
        E[0] = gather<N>(acc, 0, ss[0], su[1], su[2], ws[0], wu[1], wu[2]);
        E[1] = gather<N>(acc, 1, su[0], ss[1], su[2], wu[0], ws[1], wu[2]);
        E[2] = gather<N>(acc, 2, su[0], su[1], ss[2], wu[0], wu[1], ws[2]);
        B[0] = gather<N>(acc, 3, su[0], ss[1], ss[2], wu[0], ws[1], ws[2]);
        B[1] = gather<N>(acc, 4, ss[0], su[1], ss[2], ws[0], wu[1], ws[2]);
        B[2] = gather<N>(acc, 5, ss[0], ss[1], su[2], ws[0], ws[1], wu[2]);
        if (ext.type == PIC_EXT_PLANAR_UNDULATOR) {
            float f = 1.f;
            if (ext.ramp_mode) {
                const float r = fmaf(ext.ramp_a, (float)c[2] + o[2], ext.ramp_b);
                f = ext.ramp_mode == 1 ? fminf(fmaxf(r, 0.f), 1.f) : (r >= 0.f ? 1.f : 0.f);
            }
            const float ph = ext.phase_tab[c[2]] + fmaf(ext.kdz, o[2], ext.theta);
            const float By = ext.B0g * f * cosf(ph);
            B[1] += By;
            E[0] -= ext.beta_R * By;
        }
        // Boris rotation
        const float h = sp.h_qm;
        float um[3];
#pragma unroll
        for (int d = 0; d < 3; d++) um[d] = fmaf(h, E[d], u[d]);
        const float ig = rsqrtf(1.f + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
        float t[3];
#pragma unroll
        for (int d = 0; d < 3; d++) t[d] = h * B[d] * ig;
        const float s2 = 2.f / (1.f + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        const float up[3] = {um[0] + um[1] * t[2] - um[2] * t[1], um[1] + um[2] * t[0] - um[0] * t[2],
                             um[2] + um[0] * t[1] - um[1] * t[0]};
        const float sv[3] = {s2 * t[0], s2 * t[1], s2 * t[2]};
        u[0] = um[0] + up[1] * sv[2] - up[2] * sv[1] + h * E[0];
        u[1] = um[1] + up[2] * sv[0] - up[0] * sv[2] + h * E[1];
        u[2] = um[2] + up[0] * sv[1] - up[1] * sv[0] + h * E[2];
        mo.x = u[0]; mo.y = u[1]; mo.z = u[2];
    }
    const float ig = rsqrtf(1.f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(ig > 0.f)) { atomicOr(err, ERR_NAN); return false; }
    int s[3];
    float o1[3];
    bool alive = true;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float x1 = fmaf(u[d] * ig, g.dt_over_d[d], o[d]);
        s[d] = (int)floorf(x1);
        o1[d] = x1 - (float)s[d];
        if (o1[d] >= 1.f) { o1[d] = 0.f; s[d] += 1; }
        if (s[d] < -1 || s[d] > 1) { atomicOr(err, ERR_MOVE); return false; }
        int cn = c[d] + s[d];
        if (g.periodic[d]) {
            cn = cn < 0 ? cn + g.n[d] : (cn >= g.n[d] ? cn - g.n[d] : cn);
        } else if (cn < g.mlo || cn > g.n[d] - 1 - g.mhi) {
            alive = false;
        }
        c[d] = cn;   // new cell; the deposit below is relative to the old cell via acc
    }
    if (!alive) return false;
    int st[3];
    float S0[3][L], S1[3][L], DS[3][L];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        S::window(o[d], s[d], o1[d], st[d], S0[d], S1[d]);
#pragma unroll
        for (int a = 0; a < L; a++) DS[d][a] = S1[d][a] - S0[d][a];
    }
    const float fac[3] = {sp.cf[0] * mo.w, sp.cf[1] * mo.w, sp.cf[2] * mo.w};
    esirkepov<L>(acc, st, S0, DS, fac);
#pragma unroll
    for (int d = 0; d < 3; d++) o[d] = o1[d];
    return true;
}

template <int ORDER, bool FROZEN>
__global__ void __launch_bounds__(kPushThreads)
k_push(SpeciesDev sp, GridDev g, TileDev t, FieldsDev f, ExtDev ext, int *work, int *err)
{
    extern __shared__ float smem[];
    __shared__ int s_item;
    const int Rx = t.R[0], R2 = t.R[0] * t.R[1], R3 = R2 * t.R[2];
    float *sF = smem;
    float *sJ = FROZEN ? smem : smem + 6 * R3;
    const int n_total = sp.count[0], n_sorted = sp.count[1], n_tile_items = sp.count[2];
    const int n_items = n_tile_items + (n_total - n_sorted + kChunk - 1) / kChunk;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;

        if (item < n_tile_items) {
            const int2 it = t.items[item];
            const int tile = it.x;
            const int tx = tile % t.nt[0], ty = (tile / t.nt[0]) % t.nt[1], tz = tile / (t.nt[0] * t.nt[1]);
            const int t0[3] = {tx * t.T[0], ty * t.T[1], tz * t.T[2]};
            const int reg0[3] = {t0[0] - t.M - t.hl, t0[1] - t.M - t.hl, t0[2] - t.M - t.hl};
            const int key0 = tile * t.tile_cells;
            const int p_begin = t.cell_start[key0] + it.y * kChunk;
            const int p_end = min(p_begin + kChunk, t.cell_start[key0 + t.tile_cells]);
            // stage E/B of the region, zero the J region
            for (int l = threadIdx.x; l < (FROZEN ? 3 : 9) * R3; l += blockDim.x) {
                const int comp = l / R3, r = l - comp * R3;
                if (!FROZEN && comp < 6) {
                    const int lz = r / R2, ly = (r - lz * R2) / Rx, lx = r - lz * R2 - ly * Rx;
                    int p[3] = {reg0[0] + lx, reg0[1] + ly, reg0[2] + lz};
                    bool ok = true;
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        if (p[d] < 0 || p[d] >= g.n[d]) {
                            if (g.periodic[d]) p[d] = p[d] < 0 ? p[d] + g.n[d] : p[d] - g.n[d];
                            else ok = false;
                        }
                    }
                    float v = 0.f;
                    if (ok) {
                        const long long ix = ((long long)p[2] * g.n[1] + p[1]) * g.n[0] + p[0];
                        v = comp < 3 ? __ldg(f.E + comp * g.ncell + ix) : __ldg(f.B + (comp - 3) * g.ncell + ix);
                    }
                    sF[l] = v;
                } else {
                    sJ[l - (FROZEN ? 0 : 6 * R3)] = 0.f;
                }
            }
            __syncthreads();
            for (int p = p_begin + threadIdx.x; p < p_end; p += blockDim.x) {
                float4 P = sp.pos[p];
                const int cell = __float_as_int(P.w);
                if (cell < 0) continue;
                float4 mo = sp.mom[p];
                int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
                float o[3] = {P.x, P.y, P.z};
                int rel[3];
                bool fast = true;
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    int r = c[d] - t0[d];
                    if (g.periodic[d]) {
                        if (r > g.n[d] / 2) r -= g.n[d];
                        else if (r < -g.n[d] / 2) r += g.n[d];
                    }
                    rel[d] = r;
                    fast = fast && r >= -t.M && r < t.T[d] + t.M;
                }
                bool alive;
                if (fast) {
                    SmemAcc acc{sF, sJ, Rx, R2, R3,
                                ((rel[2] + t.M + t.hl) * t.R[1] + rel[1] + t.M + t.hl) * Rx + rel[0] + t.M + t.hl};
                    alive = advance<ORDER, FROZEN>(acc, o, c, mo, sp, g, ext, err);
                } else {
                    GlobAcc acc{f.E, f.B, f.J, g, {c[0], c[1], c[2]}, err};
                    alive = advance<ORDER, FROZEN>(acc, o, c, mo, sp, g, ext, err);
                }
                if (alive) {
                    P = make_float4(o[0], o[1], o[2], __int_as_float(pack_cell(c[0], c[1], c[2])));
                    if (!FROZEN) sp.mom[p] = mo;
                } else {
                    P.w = __int_as_float(-1);
                }
                sp.pos[p] = P;
            }
            __syncthreads();
            // one flush of the region's current to global memory
            for (int l = threadIdx.x; l < 3 * R3; l += blockDim.x) {
                const float v = sJ[l];
                if (v == 0.f) continue;
                const int comp = l / R3, r = l - comp * R3;
                const int lz = r / R2, ly = (r - lz * R2) / Rx, lx = r - lz * R2 - ly * Rx;
                int p[3] = {reg0[0] + lx, reg0[1] + ly, reg0[2] + lz};
                bool ok = true;
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    if (p[d] < 0 || p[d] >= g.n[d]) {
                        if (g.periodic[d]) p[d] = p[d] < 0 ? p[d] + g.n[d] : p[d] - g.n[d];
                        else ok = false;
                    }
                }
                if (!ok) { atomicOr(err, ERR_INDEX); continue; }
                atomicAdd(f.J + comp * g.ncell + ((long long)p[2] * g.n[1] + p[1]) * g.n[0] + p[0], v);
            }
        } else {
            const int p_begin = n_sorted + (item - n_tile_items) * kChunk;
            const int p_end = min(p_begin + kChunk, n_total);
            for (int p = p_begin + threadIdx.x; p < p_end; p += blockDim.x) {
                float4 P = sp.pos[p];
                const int cell = __float_as_int(P.w);
                if (cell < 0) continue;
                float4 mo = sp.mom[p];
                int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
                float o[3] = {P.x, P.y, P.z};
                GlobAcc acc{f.E, f.B, f.J, g, {c[0], c[1], c[2]}, err};
                const bool alive = advance<ORDER, FROZEN>(acc, o, c, mo, sp, g, ext, err);
                if (alive) {
                    P = make_float4(o[0], o[1], o[2], __int_as_float(pack_cell(c[0], c[1], c[2])));
                    if (!FROZEN) sp.mom[p] = mo;
                } else {
                    P.w = __int_as_float(-1);
                }
                sp.pos[p] = P;
            }
        }
    }
}

template <int ORDER, bool FROZEN>
cudaError_t launch_push_t(pic_ctx *c, int si, const ExtDev &ext)
{
    const Species &s = c->sp[si];
    TileDev t = tile_dev(c, s);
    const size_t smem = (size_t)(FROZEN ? 3 : 9) * t.R[0] * t.R[1] * t.R[2] * sizeof(float);
    auto kern = k_push<ORDER, FROZEN>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPushThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    FieldsDev f{c->E, c->B, c->J};
    kern<<<c->num_sms * per_sm, kPushThreads, smem, c->stream>>>(species_dev(c, s), grid_dev(c), t, f, ext,
                                                                   c->work + si, c->err);
    return cudaGetLastError();
}

// Charge density at the nodes: rho += q w S(node - x) / V for every live particle.
template <int ORDER>
__global__ void k_rho(SpeciesDev sp, GridDev g, float qv, float *rho)
{
    using S = Shape<ORDER>;
    const int n = sp.count[0];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 P = sp.pos[p];
        const int cell = __float_as_int(P.w);
        if (cell < 0) continue;
        const float w = sp.mom[p].w * qv;
        int c[3] = {cell_i(cell), cell_j(cell), cell_k(cell)};
        float o[3] = {P.x, P.y, P.z};
        int su[3];
        float wu[3][S::N];
#pragma unroll
        for (int d = 0; d < 3; d++) S::unst(o[d], su[d], wu[d]);
        for (int k = 0; k < S::N; k++)
            for (int j = 0; j < S::N; j++)
                for (int i = 0; i < S::N; i++) {
                    int q[3] = {c[0] + su[0] + i, c[1] + su[1] + j, c[2] + su[2] + k};
                    bool ok = true;
                    for (int d = 0; d < 3; d++) {
                        if (q[d] < 0 || q[d] >= g.n[d]) {
                            if (g.periodic[d]) q[d] = q[d] < 0 ? q[d] + g.n[d] : q[d] - g.n[d];
                            else ok = false;
                        }
                    }
                    if (ok)
                        atomicAdd(rho + ((long long)q[2] * g.n[1] + q[1]) * g.n[0] + q[0],
                                  w * wu[0][i] * wu[1][j] * wu[2][k]);
                }
    }
}

}  // namespace

cudaError_t launch_push(pic_ctx *c, int si, const ExtDev &ext)
{
    const bool fr = c->sp[si].frozen != 0;
    if (c->order == 1) return fr ? launch_push_t<1, true>(c, si, ext) : launch_push_t<1, false>(c, si, ext);
    return fr ? launch_push_t<2, true>(c, si, ext) : launch_push_t<2, false>(c, si, ext);
}

cudaError_t launch_rho(pic_ctx *c, float *rho)
{
    cudaError_t e = cudaMemsetAsync(rho, 0, sizeof(float) * c->ncell, c->stream);
    if (e != cudaSuccess) return e;
    const float V = (float)(c->d[0] * c->d[1] * c->d[2]);
    for (int si = 0; si < c->nsp; si++) {
        const Species &s = c->sp[si];
        const float qv = (float)(s.q / V);
        if (c->order == 1) k_rho<1><<<c->num_sms * 8, 256, 0, c->stream>>>(species_dev(c, s), grid_dev(c), qv, rho);
        else k_rho<2><<<c->num_sms * 8, 256, 0, c->stream>>>(species_dev(c, s), grid_dev(c), qv, rho);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gbpic
