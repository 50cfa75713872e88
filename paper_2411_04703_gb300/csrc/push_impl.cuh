// Fused particle kernel of one boosted-frame PIC step (sm_103a): implementation shared by the
// CIC (k_push1.cu) and TSC (k_push2.cu) translation units.
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
//
// Deposit split: a particle whose nearest node (TSC) or cell (CIC) does not change in any
// dimension during the step -- all but a few percent in a cold drifting plasma -- has its
// Esirkepov current on a window of order+1 nodes per dimension with DS in closed form
// (54 node updates for TSC instead of 144); the others are queued in shared memory and
// deposited with the general window of order+2 nodes after the main loop.
#pragma once

#include <mutex>
#include "gbpic_internal.cuh"

#include <algorithm>

namespace gbpic {
namespace push {

constexpr int kQueue = 1024;  // queued crossing particles per work item (overflow: inline)

// ------------------------------------------------------------------ region geometry
// The z-plane pitch is padded to 4 (mod 16) words.  The 32 lanes of a warp work on cells 16
// apart in the tile's (x, z, y) order, i.e. the same x, z = z0 + 2b (b < 4) and y = y0 + a
// (a < 8); their words then sit at Rx a + 2 pitch b = Rx a + 8 b (mod 32), which with an odd
// region width Rx are 32 different banks.
__host__ __device__ constexpr int plane_pitch(int rx, int ry) { return rx * ry + (((4 - (rx * ry) % 16) % 16) + 16) % 16; }

struct RegDyn {
    int Rx, Ry, R2, R3;   // R2: padded plane pitch; R3 = R2 * Rz
    __device__ __forceinline__ int rx() const { return Rx; }
    __device__ __forceinline__ int ry() const { return Ry; }
    __device__ __forceinline__ int r2() const { return R2; }
    __device__ __forceinline__ int r3() const { return R3; }
};
template <int RX, int RY, int RZ> struct RegFix {
    __device__ __forceinline__ static constexpr int rx() { return RX; }
    __device__ __forceinline__ static constexpr int ry() { return RY; }
    __device__ __forceinline__ static constexpr int r2() { return plane_pitch(RX, RY); }
    __device__ __forceinline__ static constexpr int r3() { return plane_pitch(RX, RY) * RZ; }
};

// ------------------------------------------------------------------ shape weights
// Shape S of order 1 (CIC) or 2 (TSC).  Gather weights on the integer nodes (unst) and on the
// half-integer nodes m + 1/2 (stag), given the in-cell offset o of cell c: nodes start at c + s.
//
// General deposit weights: S0 = S(node - x^n) and DS = S(node - x^{n+1}) - S(node - x^n) on a
// window of L nodes starting at c + st.  DS is formed without subtracting two shape values:
// with the displacement d of the push, DS(m) = integral of S' over [t0, t0 + d] (t0 = o - m),
// split at the knot of S that the segment crosses; S' is constant (CIC) or linear (TSC) on each
// piece, so piece = length * S'(midpoint) is exact, and the length before the knot is taken in
// offset space, (m + k) - o, which is exact near a crossing.  A slow component (|d| << 1 cell)
// thus keeps full FP32 relative precision in its current.
template <int ORDER> struct Shape;

// Order 0 (nearest grid point), used only by the energy-conserving gather of the first-order
// shape along a staggered dim: the half-integer node nearest to the offset o in [0, 1) is c + 1/2
// (c - 1/2 when o = 0, the half-open convention of the shape).
template <> struct Shape<0> {
    static constexpr int N = 1;
    __device__ __forceinline__ static void stag(float o, int &s, float w[1]) {
        s = o > 0.f ? 0 : -1; w[0] = 1.f;
    }
};

template <> struct Shape<1> {
    static constexpr int N = 2;   // gather nodes per dim
    static constexpr int L = 3;   // general Esirkepov window per dim
    __device__ __forceinline__ static void unst(float o, int &s, float w[2]) {
        s = 0; w[0] = 1.f - o; w[1] = o;
    }
    __device__ __forceinline__ static void stag(float o, int &s, float w[2]) {
        const bool hi = o >= 0.5f;
        const float f = hi ? o - 0.5f : o + 0.5f;
        s = hi ? 0 : -1; w[0] = 1.f - f; w[1] = f;
    }
    __device__ __forceinline__ static float S(float t) { return fmaxf(0.f, 1.f - fabsf(t)); }
    __device__ __forceinline__ static float dS(float t) {
        return fabsf(t) < 1.f ? (t > 0.f ? -1.f : (t < 0.f ? 1.f : 0.f)) : 0.f;
    }
    __device__ __forceinline__ static float seg(float o, int m, float d) {
        const float t0 = o - (float)m, t1 = t0 + d;
        const float lo = fminf(t0, t1), hi = fmaxf(t0, t1);
        const float k = ceilf(hi) - 1.f;            // largest knot below hi
        if (!(k > lo)) return d * dS(t0 + 0.5f * d);
        const float a = ((float)m + k) - o;
        return a * dS(k - 0.5f * a) + (d - a) * dS(k + 0.5f * (d - a));
    }
    __device__ __forceinline__ static void general(float o, float d, int s, int &st, float S0[3], float DS[3]) {
        st = min(s, 0);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            S0[a] = S(o - (float)(st + a));
            DS[a] = seg(o, st + a, d);
        }
    }
    // the cell does not change: window {c, c+1}
    __device__ __forceinline__ static bool stays(float o, float d, int s) { return s == 0; }
    __device__ __forceinline__ static void simple(float o, float d, int &st, float S0[2], float DS[2]) {
        st = 0;
        S0[0] = 1.f - o; S0[1] = o;
        DS[0] = -d; DS[1] = d;
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
    __device__ __forceinline__ static float S(float t) {
        const float a = fabsf(t);
        return a <= 0.5f ? 0.75f - a * a : (a < 1.5f ? 0.5f * (1.5f - a) * (1.5f - a) : 0.f);
    }
    __device__ __forceinline__ static float dS(float t) {
        const float a = fabsf(t);
        const float v = a <= 0.5f ? -2.f * a : (a < 1.5f ? a - 1.5f : 0.f);
        return t < 0.f ? -v : v;
    }
    __device__ __forceinline__ static float seg(float o, int m, float d) {
        const float t0 = o - (float)m, t1 = t0 + d;
        const float lo = fminf(t0, t1), hi = fmaxf(t0, t1);
        const float k = ceilf(hi - 0.5f) - 0.5f;    // largest knot below hi
        if (!(k > lo)) return d * dS(t0 + 0.5f * d);
        const float a = ((float)m + k) - o;
        return a * dS(k - 0.5f * a) + (d - a) * dS(k + 0.5f * (d - a));
    }
    __device__ __forceinline__ static void general(float o, float d, int /*s*/, int &st, float S0[4], float DS[4]) {
        const int b0 = o >= 0.5f;
        const int b1 = (int)floorf(o + d + 0.5f);   // nearest node of the new position, rel. to c
        st = b0 - 1 + min(b1 - b0, 0);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            S0[a] = S(o - (float)(st + a));
            DS[a] = seg(o, st + a, d);
        }
    }
    // the nearest node does not change: window {b-1, b, b+1}; with dl = o - b in [-1/2, 1/2),
    // S0 = TSC weights of dl and DS in closed form (each node stays on one polynomial piece)
    __device__ __forceinline__ static bool stays(float o, float d, int) {
        return (int)floorf(o + d + 0.5f) == (int)(o >= 0.5f);
    }
    __device__ __forceinline__ static void simple(float o, float d, int &st, float S0[3], float DS[3]) {
        const int b = o >= 0.5f;
        const float dl = o - (float)b;
        st = b - 1;
        tsc(dl, S0);
        DS[0] = -d * (0.5f - dl - 0.5f * d);
        DS[1] = -d * (2.f * dl + d);
        DS[2] = d * (0.5f + dl + 0.5f * d);
    }
};

// ------------------------------------------------------------------ field / current access
// Shared-memory region of a tile: node (c + x) of the particle's cell c sits at local linear
// index base + x + y Rx + z Rx Ry.
//
// The region's current is accumulated as exact fixed point with native 32-bit integer shared
// atomics (a float add on shared memory is not a native atomic): a contribution v becomes
// V = round(v * js), an int32 with |V| <= 2^30 for the largest contribution the work item can
// receive (largest weight of the run, charge, and the step's displacement bound dlim), split into
// its 19 low bits (unsigned word) and the rest (signed word).  js is a power of two, so the flush
// (hi * 2^19 + lo) / js is exact.  A work item holds at most kChunk = 4096 particles, each adding
// at most once per node and component, so neither word overflows.  dlim adapts each step to
// four times the largest displacement of the previous one, so a slow current component (a plasma's
// transverse motion) keeps its precision; a particle moving further than dlim deposits with
// float atomics instead.
constexpr int kLoBits = 19;
constexpr unsigned kLoMask = (1u << kLoBits) - 1u;
static_assert(kChunk <= 4096, "fixed-point current words sized for 4096 contributions per node");

template <class Reg> struct SmemAcc {
    Reg reg;
    const float *sF;
    unsigned *sJlo;
    int *sJhi;
    const float *js;      // shared [3]: fixed-point scale of the work item
    int base;
    __device__ __forceinline__ float scale(int comp) const { return js[comp]; }
    __device__ __forceinline__ float f(int comp, int x, int y, int z) const {
        return sF[comp * reg.r3() + base + z * reg.r2() + y * reg.rx() + x];
    }
    // v is already in fixed-point units (times scale(comp)), |v| <= 2^30
    __device__ __forceinline__ void j(int comp, int x, int y, int z, float v) const {
        const int ix = comp * reg.r3() + base + z * reg.r2() + y * reg.rx() + x;
        const int V = __float2int_rn(v);
        atomicAdd(&sJlo[ix], (unsigned)V & kLoMask);
        atomicAdd(&sJhi[ix], V >> kLoBits);
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
    int zb;               // first row of the particle's run
    __device__ __forceinline__ long long node(int x, int y, int z) const {
        int p[3] = {c[0] + x, c[1] + y, c[2] + z};
#pragma unroll
        for (int d = 0; d < 2; d++) {
            if (p[d] < 0 || p[d] >= g.n[d]) {
                if (!g.periodic[d]) return -1;
                p[d] = pwrap(p[d], g.n[d]);
            }
        }
        if (p[2] < zb || p[2] >= zb + g.nzr) {
            if (!g.periodic[2]) return -1;
            p[2] = zb + pwrap(p[2] - zb, g.nzr);
        }
        return ((long long)p[2] * g.n[1] + p[1]) * g.n[0] + p[0];
    }
    __device__ __forceinline__ float scale(int) const { return 1.f; }
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

template <int NX, int NY, int NZ, class Acc>
__device__ __forceinline__ float gather3(const Acc &a, int comp, int sx, int sy, int sz,
                                         const float *wx, const float *wy, const float *wz)
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NZ; k++) {
        float sk = 0.f;
#pragma unroll
        for (int j = 0; j < NY; j++) {
            float sj = 0.f;
#pragma unroll
            for (int i = 0; i < NX; i++) sj = fmaf(wx[i], a.f(comp, sx + i, sy + j, sz + k), sj);
            sk = fmaf(wy[j], sj, sk);
        }
        s = fmaf(wz[k], sk, s);
    }
    return s;
}

template <int N, class Acc>
__device__ __forceinline__ float gather(const Acc &a, int comp, int sx, int sy, int sz,
                                        const float *wx, const float *wy, const float *wz)
{
    return gather3<N, N, N>(a, comp, sx, sy, sz, wx, wy, wz);
}

// ------------------------------------------------------------------ Esirkepov
// W_c = DS_c (S0_a S0_b + DS_a S0_b/2 + S0_a DS_b/2 + DS_a DS_b/3) for the two other dims a, b,
// written as DS_c [A_a A_b + DS_a DS_b / 12] with A = S0 + DS/2, and J_c(node + 1/2) =
// -q w (d_c/dt) (sum of W_c over the nodes up to this one) / V; the prefix over the last window
// node vanishes (sum DS = 0) and is not stored.  fac = -q w d_c/(dt V).
template <int L, bool TEST_ZERO, class Acc>
__device__ __forceinline__ void esirkepov(const Acc &acc, const int st[3], const float S0[3][L],
                                          const float DS[3][L], const float fac[3], bool skip_x, bool skip_y)
{
    float A[3][L], Q[3][L];
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int a = 0; a < L; a++) {
            A[d][a] = fmaf(0.5f, DS[d][a], S0[d][a]);
            Q[d][a] = DS[d][a] * (1.f / 12.f);
        }
    float P[3][L - 1];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float fs = fac[d] * acc.scale(d);
        float run = 0.f;
#pragma unroll
        for (int a = 0; a < L - 1; a++) {
            run += DS[d][a];
            P[d][a] = fs * run;
        }
    }
    if (!skip_x) {
#pragma unroll
        for (int k = 0; k < L; k++)
#pragma unroll
            for (int j = 0; j < L; j++) {
                const float Y = fmaf(A[1][j], A[2][k], Q[1][j] * DS[2][k]);
                if (TEST_ZERO && Y == 0.f) continue;
#pragma unroll
                for (int i = 0; i < L - 1; i++)
                    if (!TEST_ZERO || P[0][i] != 0.f) acc.j(0, st[0] + i, st[1] + j, st[2] + k, P[0][i] * Y);
            }
    }
    if (!skip_y) {
#pragma unroll
        for (int k = 0; k < L; k++)
#pragma unroll
            for (int i = 0; i < L; i++) {
                const float Y = fmaf(A[2][k], A[0][i], Q[2][k] * DS[0][i]);
                if (TEST_ZERO && Y == 0.f) continue;
#pragma unroll
                for (int j = 0; j < L - 1; j++)
                    if (!TEST_ZERO || P[1][j] != 0.f) acc.j(1, st[0] + i, st[1] + j, st[2] + k, P[1][j] * Y);
            }
    }
#pragma unroll
    for (int j = 0; j < L; j++)
#pragma unroll
        for (int i = 0; i < L; i++) {
            const float Y = fmaf(A[0][i], A[1][j], Q[0][i] * DS[1][j]);
            if (TEST_ZERO && Y == 0.f) continue;
#pragma unroll
            for (int k = 0; k < L - 1; k++)
                if (!TEST_ZERO || P[2][k] != 0.f) acc.j(2, st[0] + i, st[1] + j, st[2] + k, P[2][k] * Y);
        }
}

// General window (order+2 nodes per dim), any move below one cell.
template <int ORDER, class Acc>
__device__ __forceinline__ void deposit_general(const Acc &acc, const float o[3], const float d[3],
                                                const int s[3], const float fac[3])
{
    using S = Shape<ORDER>;
    constexpr int L = S::L;
    int st[3];
    float S0[3][L], DS[3][L];
#pragma unroll
    for (int dd = 0; dd < 3; dd++) S::general(o[dd], d[dd], s[dd], st[dd], S0[dd], DS[dd]);
    esirkepov<L, true>(acc, st, S0, DS, fac, d[0] == 0.f, d[1] == 0.f);
}

// Nearest node / cell unchanged in every dimension: window of order+1 nodes.
template <int ORDER, class Acc>
__device__ __forceinline__ void deposit_simple(const Acc &acc, const float o[3], const float d[3],
                                               const float fac[3])
{
    using S = Shape<ORDER>;
    constexpr int L = S::N;
    int st[3];
    float S0[3][L], DS[3][L];
#pragma unroll
    for (int dd = 0; dd < 3; dd++) S::simple(o[dd], d[dd], st[dd], S0[dd], DS[dd]);
    esirkepov<L, false>(acc, st, S0, DS, fac, d[0] == 0.f, d[1] == 0.f);
}

// Gather, external field and Boris rotation of one particle: u^{n-1/2} -> u^{n+1/2} in mo.
// GATHER 0: momentum-conserving (the deposit's shape at each component's Yee point); GATHER 1:
// energy-conserving (one order lower along the component's staggered dims: the transpose of the
// Esirkepov deposit, whose J_x has the lower-order shape at the half-integer x nodes).
template <int ORDER, class Acc, int GATHER = 0>
__device__ __forceinline__ void push_u(const Acc &acc, const float o[3], const int c[3], float4 &mo,
                                       const SpeciesDev &sp, const ExtDev &ext)
{
    using S = Shape<ORDER>;
    using SS = Shape<GATHER ? ORDER - 1 : ORDER>;   // shape along staggered dims
    constexpr int N = S::N, NS = SS::N;
    int su[3], ss[3];
    float wu[3][N], ws[3][NS];
#pragma unroll
    for (int dd = 0; dd < 3; dd++) { S::unst(o[dd], su[dd], wu[dd]); SS::stag(o[dd], ss[dd], ws[dd]); }
    float E[3], B[3];
    E[0] = gather3<NS, N, N>(acc, 0, ss[0], su[1], su[2], ws[0], wu[1], wu[2]);
    E[1] = gather3<N, NS, N>(acc, 1, su[0], ss[1], su[2], wu[0], ws[1], wu[2]);
    E[2] = gather3<N, N, NS>(acc, 2, su[0], su[1], ss[2], wu[0], wu[1], ws[2]);
    B[0] = gather3<N, NS, NS>(acc, 3, su[0], ss[1], ss[2], wu[0], ws[1], ws[2]);
    B[1] = gather3<NS, N, NS>(acc, 4, ss[0], su[1], ss[2], ws[0], wu[1], ws[2]);
    B[2] = gather3<NS, NS, N>(acc, 5, ss[0], ss[1], su[2], ws[0], ws[1], wu[2]);
    if (ext.type == PIC_EXT_PLANAR_UNDULATOR || ext.type == PIC_EXT_PLANAR_UNDULATOR_3D) {
        float f = 1.f;
        if (ext.ramp_mode) {
            const float r = fmaf(ext.ramp_a, (float)c[2] + o[2], ext.ramp_b);
            f = ext.ramp_mode == 1 ? fminf(fmaxf(r, 0.f), 1.f) : (r >= 0.f ? 1.f : 0.f);
        }
        const float ph = ext.phase_tab[c[2]] + fmaf(ext.kdz, o[2], ext.theta);
        const float amp = (ext.amp_tab ? __ldg(ext.amp_tab + c[2]) : ext.B0g) * f;
        float By = amp * cosf(ph);
        if (ext.type == PIC_EXT_PLANAR_UNDULATOR_3D) {
            // k_u y from the axis; B'_z = B_z is the lab amplitude (B'_y's over gamma_R)
            const float ky = ((float)c[1] - ext.y0 + o[1]) * ext.kuy;
            B[2] -= amp * ext.igR * sinhf(ky) * sinf(ph);
            By *= coshf(ky);
        }
        B[1] += By;
        E[0] -= ext.beta_R * By;
    }
    const float h = sp.h_qm;
    if (sp.pusher == PIC_PUSHER_VAY) {
        // Vay: half kick with the old velocity, then the rotation whose Lorentz factor solves
        // gamma^2 = (sigma + sqrt(sigma^2 + 4 (tau^2 + (u'.tau)^2))) / 2
        const float u0[3] = {mo.x, mo.y, mo.z};
        const float ig0 = rsqrtf(1.f + u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2]);
        const float v[3] = {u0[0] * ig0, u0[1] * ig0, u0[2] * ig0};
        const float vxb[3] = {v[1] * B[2] - v[2] * B[1], v[2] * B[0] - v[0] * B[2], v[0] * B[1] - v[1] * B[0]};
        float up[3], tau[3];
#pragma unroll
        for (int dd = 0; dd < 3; dd++) {
            up[dd] = u0[dd] + h * (E[dd] + vxb[dd]) + h * E[dd];
            tau[dd] = h * B[dd];
        }
        const float tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
        const float ust = up[0] * tau[0] + up[1] * tau[1] + up[2] * tau[2];
        const float sig = 1.f + up[0] * up[0] + up[1] * up[1] + up[2] * up[2] - tau2;
        const float ig1 = rsqrtf(0.5f * (sig + sqrtf(sig * sig + 4.f * (tau2 + ust * ust))));
        const float t[3] = {tau[0] * ig1, tau[1] * ig1, tau[2] * ig1};
        const float s = 1.f / (1.f + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        const float ut = up[0] * t[0] + up[1] * t[1] + up[2] * t[2];
        mo.x = s * (up[0] + ut * t[0] + up[1] * t[2] - up[2] * t[1]);
        mo.y = s * (up[1] + ut * t[1] + up[2] * t[0] - up[0] * t[2]);
        mo.z = s * (up[2] + ut * t[2] + up[0] * t[1] - up[1] * t[0]);
        return;
    }
    float um[3];
#pragma unroll
    for (int dd = 0; dd < 3; dd++) um[dd] = fmaf(h, E[dd], dd == 0 ? mo.x : (dd == 1 ? mo.y : mo.z));
    const float ig = rsqrtf(1.f + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    float t[3];
#pragma unroll
    for (int dd = 0; dd < 3; dd++) t[dd] = h * B[dd] * ig;
    const float s2 = 2.f / (1.f + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    const float up[3] = {um[0] + um[1] * t[2] - um[2] * t[1], um[1] + um[2] * t[0] - um[0] * t[2],
                         um[2] + um[0] * t[1] - um[1] * t[0]};
    const float sv[3] = {s2 * t[0], s2 * t[1], s2 * t[2]};
    mo.x = um[0] + up[1] * sv[2] - up[2] * sv[1] + h * E[0];
    mo.y = um[1] + up[2] * sv[0] - up[0] * sv[2] + h * E[1];
    mo.z = um[2] + up[0] * sv[1] - up[1] * sv[0] + h * E[2];
}

// Gather, external field, Boris push (unless FROZEN) and move of one particle.  On return d
// holds the push displacement (cells), s the cell shift, o1 the new offsets and c the new cell.
// Returns false when the particle left through a non-periodic face (it becomes a dummy).
template <int ORDER, bool FROZEN, class Acc, int GATHER = 0>
__device__ __forceinline__ bool push_move(const Acc &acc, const float o[3], int c[3], float4 &mo,
                                          const SpeciesDev &sp, const GridDev &g, const ExtDev &ext,
                                          int *err, float d[3], int s[3], float o1[3], int zb)
{
    if (!FROZEN) push_u<ORDER, Acc, GATHER>(acc, o, c, mo, sp, ext);
    const float u[3] = {mo.x, mo.y, mo.z};
    const float ig = rsqrtf(1.f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(ig > 0.f)) { atomicOr(err, ERR_NAN); return false; }
    bool alive = true;
#pragma unroll
    for (int dd = 0; dd < 3; dd++) {
        d[dd] = u[dd] * ig * g.dt_over_d[dd];        // displacement of the push (cells)
        const float x1 = o[dd] + d[dd];
        s[dd] = (int)floorf(x1);
        o1[dd] = x1 - (float)s[dd];
        if (o1[dd] >= 1.f) { o1[dd] = 0.f; s[dd] += 1; }
        if (s[dd] < -1 || s[dd] > 1) { atomicOr(err, ERR_MOVE); return false; }
        int cn = c[dd] + s[dd];
        if (g.periodic[dd]) {
            cn = dd == 2 ? zwrap(cn, zb, g.nzr) : (cn < 0 ? cn + g.n[dd] : (cn >= g.n[dd] ? cn - g.n[dd] : cn));
        } else if (cn < g.mlo || cn > g.n[dd] - 1 - g.mhi) {
            alive = false;
        }
        c[dd] = cn;
    }
    return alive;
}

template <int ORDER>
__device__ __forceinline__ bool stays_all(const float o[3], const float d[3], const int s[3])
{
    return Shape<ORDER>::stays(o[0], d[0], s[0]) && Shape<ORDER>::stays(o[1], d[1], s[1]) &&
           Shape<ORDER>::stays(o[2], d[2], s[2]);
}

// Whole step of one particle on the global-memory path.
template <int ORDER, bool FROZEN, int GATHER = 0>
__device__ __forceinline__ void step_global(const SpeciesDev &sp, const GridDev &g, const FieldsDev &f,
                                            const ExtDev &ext, int *err, int p)
{
    float4 P = sp.pos[p];
    const int cell = __float_as_int(P.w);
    if (cell < 0) return;
    float4 mo = sp.mom[p];
    int c[3] = {g.cc.i(cell), g.cc.j(cell), g.cc.k(cell)};
    const float o[3] = {P.x, P.y, P.z};
    const int zb = g.nzr == g.n[2] ? 0 : zblock(c[2], g.nzr);
    GlobAcc acc{f.E, f.B, f.J, g, {c[0], c[1], c[2]}, err, zb};
    float d[3], o1[3];
    int s[3];
    if (push_move<ORDER, FROZEN, GlobAcc, GATHER>(acc, o, c, mo, sp, g, ext, err, d, s, o1, zb)) {
        const float fac[3] = {sp.cf[0] * mo.w, sp.cf[1] * mo.w, sp.cf[2] * mo.w};
        deposit_general<ORDER>(acc, o, d, s, fac);
        P = make_float4(o1[0], o1[1], o1[2], __int_as_float(g.cc.pack(c[0], c[1], c[2])));
        if (!FROZEN) sp.mom[p] = mo;
    } else {
        P.w = __int_as_float(-1);
    }
    sp.pos[p] = P;
}

// Linear index of grid node (x, y, z) with periodic wrap (z inside the run starting at row zb),
// or -1 outside a non-periodic face.
__device__ __forceinline__ long long wrap_node(const GridDev &g, int x, int y, int z, int zb);

// Stage the six field components of a tile's region in shared memory.  A tile away from every
// face needs no wrap or bounds test; the loop runs over the region's nodes with compile-time
// divisions (fixed region) and each thread moves all components of its node.
template <class Reg>
__device__ __forceinline__ void stage_fields(const Reg &reg, const GridDev &g, const FieldsDev &f, float *sF,
                                             const int reg0[3], bool interior, long long gbase, int zb)
{
    const int Rx = reg.rx(), Ry = reg.ry(), R2 = reg.r2(), R3 = reg.r3();
    const long long gnx = g.n[0], gnxy = (long long)g.n[0] * g.n[1];
    for (int l = threadIdx.x; l < R3; l += blockDim.x) {
        const int lz = l / R2, rem = l - lz * R2, ly = rem / Rx, lx = rem - ly * Rx;
        if (ly >= Ry) continue;   // plane padding
        const long long gi = interior ? gbase + lz * gnxy + ly * gnx + lx
                                      : wrap_node(g, reg0[0] + lx, reg0[1] + ly, reg0[2] + lz, zb);
#pragma unroll
        for (int comp = 0; comp < 3; comp++) {
            sF[comp * R3 + l] = gi >= 0 ? __ldg(f.E + comp * g.ncell + gi) : 0.f;
            sF[(comp + 3) * R3 + l] = gi >= 0 ? __ldg(f.B + comp * g.ncell + gi) : 0.f;
        }
    }
}


__device__ __forceinline__ long long wrap_node(const GridDev &g, int x, int y, int z, int zb)
{
    int p[3] = {x, y, z};
#pragma unroll
    for (int d = 0; d < 2; d++) {
        if (p[d] < 0 || p[d] >= g.n[d]) {
            if (!g.periodic[d]) return -1;
            p[d] = pwrap(p[d], g.n[d]);
        }
    }
    if (p[2] < zb || p[2] >= zb + g.nzr) {
        if (!g.periodic[2]) return -1;
        p[2] = zb + pwrap(p[2] - zb, g.nzr);
    }
    return ((long long)p[2] * g.n[1] + p[1]) * g.n[0] + p[0];
}

// One CTA of kPushThreads per SM: the shared region of a tile holds most of the SM's shared
// memory, and 1024 threads at 64 registers (a few spills) hide more latency than 512 at 122.
template <int ORDER, bool FROZEN, class Reg, int GATHER>
__global__ void __launch_bounds__(kPushThreads, 1)
k_push(SpeciesDev sp, GridDev g, TileDev t, FieldsDev f, ExtDev ext0, int *work, int *work_sparse, int *err, Reg reg)
{
    const ExtDev ext = ext_at_clock(ext0);
    extern __shared__ float smem[];
    __shared__ int s_item, s_qn;
    __shared__ float s_js[3], s_jinv[3], s_dl[3];
    __shared__ unsigned s_dm[3];
    const int Rx = reg.rx(), R3 = reg.r3();
    float *sF = smem;
    unsigned *sJlo = reinterpret_cast<unsigned *>(FROZEN ? smem : smem + 6 * R3);
    int *sJhi = reinterpret_cast<int *>(sJlo + 3 * R3);
    int *qb = sJhi + 3 * R3;                              // queue: local base index
    float *qd = reinterpret_cast<float *>(qb + kQueue);  // queue: o[3], d[3], w (SoA)
    const int n_total = sp.count[0], n_sorted = sp.count[1], n_tile_items = sp.count[2];
    const int chunk = t.chunk;
    const int n_items = n_tile_items + (n_total - n_sorted + chunk - 1) / chunk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;

        if (item >= n_tile_items) {
            const int p_begin = n_sorted + (item - n_tile_items) * chunk;
            const int p_end = min(p_begin + chunk, n_total);
            for (int p = p_begin + threadIdx.x; p < p_end; p += blockDim.x)
                step_global<ORDER, FROZEN, GATHER>(sp, g, f, ext, err, p);
            continue;
        }

        const int2 wi = t.items[item];
        const int tile = wi.x;
        const int tx = tile % t.nt[0], ty = (tile / t.nt[0]) % t.nt[1], tz = tile / (t.nt[0] * t.nt[1]);
        const int t0[3] = {tx * t.T[0], ty * t.T[1], tz * t.T[2]};
        const int reg0[3] = {t0[0] - t.M - t.hl, t0[1] - t.M - t.hl, t0[2] - t.M - t.hl};
        const int p_begin = t.tile_start[tile] + wi.y * chunk;
        const int p_end = min(p_begin + chunk, t.tile_start[tile + 1]);
        // Region of the tile: nodes reg0 + (0..R-1) per dim (plane pitch padded).
        const int R2 = reg.r2(), Ry = reg.ry(), Rz = R3 / R2;
        const int zb = g.nzr == g.n[2] ? 0 : zblock(t0[2], g.nzr);   // the tile's run (tiles never straddle runs)
        const bool interior = reg0[0] >= 0 && reg0[0] + Rx <= g.n[0] && reg0[1] >= 0 && reg0[1] + Ry <= g.n[1] &&
                              reg0[2] >= zb && reg0[2] + Rz <= zb + g.nzr;
        const long long gnx = g.n[0], gnxy = (long long)g.n[0] * g.n[1];
        const long long gbase = reg0[2] * gnxy + reg0[1] * gnx + reg0[0];
        if (!FROZEN) stage_fields(reg, g, f, sF, reg0, interior, gbase, zb);
        for (int l = threadIdx.x; l < 3 * R3; l += blockDim.x) {
            sJlo[l] = 0u;
            sJhi[l] = 0;
        }
        if (threadIdx.x == 0) {
            s_qn = 0;
            // fixed-point scale of this item: the largest contribution jb w dlim maps to <= 2^30
            const float w = sp.wrun ? sp.wrun[t0[2] / g.nzr] : sp.wmax;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float dl = sp.dlim[k];
                const float b = sp.jb[k] * w * dl;
                int e = 0;
                frexpf(b, &e);                       // b < 2^e
                const int ex = b > 0.f ? min(max(30 - e, -100), 100) : 0;
                s_js[k] = ldexpf(1.f, ex);
                s_jinv[k] = ldexpf(1.f, -ex);
                s_dl[k] = dl;
                s_dm[k] = 0u;
            }
        }
        __syncthreads();
        // each lane takes gq consecutive particles (kGroup = 4 for a full item: half a cell of an
        // 8-per-cell lattice, visited in octant order), and a warp's lanes sit NW * gq = 128
        // particles (16 cells of that lattice) apart, so at every iteration the 32 lanes sit on 32
        // different cells with the same stencil shift (bank-conflict-free shared accesses, see
        // plane_pitch); a shorter item gives every lane fewer particles rather than idle lanes
        const int len = p_end - p_begin;
        const int gq = (len + kPushThreads - 1) / kPushThreads;
        constexpr int NW = kPushThreads / 32;
        for (int k_it = 0; k_it < gq; k_it++) {
            // lane-major: a warp's lanes sit far apart in the cell-sorted item, so in a dense bunch
            // (hundreds of particles per cell and octant) they still deposit into different
            // windows instead of queueing on the same shared-memory words; each lane's gq
            // consecutive particles share cache lines across the warps
            const int q = gq == 1 ? (int)threadIdx.x : lane * (NW * gq) + warp * gq + k_it;
            unsigned dm[3] = {0u, 0u, 0u};   // |displacement| of this lane's particle (float bits)
            do {
            if (q >= len) break;
            const int p = p_begin + q;
            float4 P = sp.pos[p];
            const int cell = __float_as_int(P.w);
            if (cell < 0) break;
            int c[3] = {g.cc.i(cell), g.cc.j(cell), g.cc.k(cell)};
            int rel[3];
            bool fast = true;
#pragma unroll
            for (int dd = 0; dd < 3; dd++) {
                int r = c[dd] - t0[dd];
                if (g.periodic[dd]) {
                    const int per = dd == 2 ? g.nzr : g.n[dd];
                    if (r > per / 2) r -= per;
                    else if (r < -per / 2) r += per;
                }
                rel[dd] = r;
                fast = fast && r >= -t.M && r < t.T[dd] + t.M;
            }
            if (!fast) {
                step_global<ORDER, FROZEN, GATHER>(sp, g, f, ext, err, p);
                break;
            }
            float4 mo = sp.mom[p];
            const float o[3] = {P.x, P.y, P.z};
            const int base = (rel[2] + t.M + t.hl) * reg.r2() + (rel[1] + t.M + t.hl) * Rx + rel[0] + t.M + t.hl;
            SmemAcc<Reg> acc{reg, sF, sJlo, sJhi, s_js, base};
            float d[3], o1[3];
            int s[3];
            if (push_move<ORDER, FROZEN, SmemAcc<Reg>, GATHER>(acc, o, c, mo, sp, g, ext, err, d, s, o1, zb)) {
                const float fac[3] = {sp.cf[0] * mo.w, sp.cf[1] * mo.w, sp.cf[2] * mo.w};
#pragma unroll
                for (int k = 0; k < 3; k++) dm[k] = __float_as_uint(fabsf(d[k]));
                if (!(fabsf(d[0]) <= s_dl[0] && fabsf(d[1]) <= s_dl[1] && fabsf(d[2]) <= s_dl[2])) {
                    // beyond the item's fixed-point range: float atomics on the global current
                    GlobAcc gacc{f.E, f.B, f.J, g, {g.cc.i(cell), g.cc.j(cell), g.cc.k(cell)}, err, zb};
                    deposit_general<ORDER>(gacc, o, d, s, fac);
                    atomicAdd(sp.nfall, 1ull);
                } else if (stays_all<ORDER>(o, d, s)) {
                    deposit_simple<ORDER>(acc, o, d, fac);
                } else {
                    const int slot = atomicAdd(&s_qn, 1);
                    if (slot < kQueue) {
                        qb[slot] = base;
                        qd[0 * kQueue + slot] = o[0];
                        qd[1 * kQueue + slot] = o[1];
                        qd[2 * kQueue + slot] = o[2];
                        qd[3 * kQueue + slot] = d[0];
                        qd[4 * kQueue + slot] = d[1];
                        qd[5 * kQueue + slot] = d[2];
                        qd[6 * kQueue + slot] = mo.w;
                    } else {
                        deposit_general<ORDER>(acc, o, d, s, fac);
                    }
                }
                P = make_float4(o1[0], o1[1], o1[2], __int_as_float(g.cc.pack(c[0], c[1], c[2])));
                if (!FROZEN) sp.mom[p] = mo;
            } else {
                P.w = __int_as_float(-1);
            }
            sp.pos[p] = P;
            } while (false);
            // the step's largest displacement per component (sets the next step's bound)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const unsigned m = __reduce_max_sync(0xffffffffu, dm[k]);
                if (lane == 0 && m) atomicMax(&s_dm[k], m);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; k++)
                if (s_dm[k]) atomicMax(sp.dmax + k, s_dm[k]);
        // queued particles that crossed a node: general window
        const int qn = min(s_qn, kQueue);
        for (int q = threadIdx.x; q < qn; q += blockDim.x) {
            const float o[3] = {qd[q], qd[kQueue + q], qd[2 * kQueue + q]};
            const float d[3] = {qd[3 * kQueue + q], qd[4 * kQueue + q], qd[5 * kQueue + q]};
            const float w = qd[6 * kQueue + q];
            int s[3];
#pragma unroll
            for (int dd = 0; dd < 3; dd++) {
                const float x1 = o[dd] + d[dd];
                s[dd] = (int)floorf(x1);
                if (x1 - (float)s[dd] >= 1.f) s[dd] += 1;
            }
            const float fac[3] = {sp.cf[0] * w, sp.cf[1] * w, sp.cf[2] * w};
            SmemAcc<Reg> acc{reg, sF, sJlo, sJhi, s_js, qb[q]};
            deposit_general<ORDER>(acc, o, d, s, fac);
        }
        __syncthreads();
        // one flush of the region's current to global memory: hi 2^19 + lo back to float
        const float jinv[3] = {s_jinv[0], s_jinv[1], s_jinv[2]};
        for (int l = threadIdx.x; l < R3; l += blockDim.x) {
            const int lz = l / R2, rem = l - lz * R2, ly = rem / Rx, lx = rem - ly * Rx;
            if (ly >= Ry) continue;   // plane padding (never written by a particle)
            long long gi = -1;
            bool have = false;
            for (int comp = 0; comp < 3; comp++) have = have || sJlo[comp * R3 + l] != 0u || sJhi[comp * R3 + l] != 0;
            if (!have) continue;
            gi = interior ? gbase + lz * gnxy + ly * gnx + lx : wrap_node(g, reg0[0] + lx, reg0[1] + ly, reg0[2] + lz, zb);
            if (gi < 0) { atomicOr(err, ERR_INDEX); continue; }
            for (int comp = 0; comp < 3; comp++) {
                const unsigned lo = sJlo[comp * R3 + l];
                const int hi = sJhi[comp * R3 + l];
                if (lo == 0u && hi == 0) continue;
                const float v = fmaf((float)hi, (float)(1u << kLoBits), __uint2float_rn(lo)) * jinv[comp];
                atomicAdd(f.J + comp * g.ncell + gi, v);
            }
        }
    }
    // sparse tiles (fewer than kSparse particles): staging and flushing a region would cost more
    // than the global-memory path of their few particles; each warp takes whole tiles
    const int n_sparse = sp.count[3];
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(work_sparse, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_sparse) break;
        const int tile = t.sparse_tiles[it];
        const int pe = t.tile_start[tile + 1];
        for (int p = t.tile_start[tile] + lane; p < pe; p += 32) step_global<ORDER, FROZEN, GATHER>(sp, g, f, ext, err, p);
    }
}

// Next step's displacement bound per component: four times the largest displacement of this step,
// within [light * 2^-10, light] (light: the speed-of-light bound); the measurement restarts.
static __global__ void k_dlim_update(float *dlim, unsigned *dmax, float l0, float l1, float l2)
{
    const int k = threadIdx.x;
    if (k >= 3) return;
    const float light = k == 0 ? l0 : (k == 1 ? l1 : l2);
    const float m = __uint_as_float(dmax[k]);
    dlim[k] = fminf(light, fmaxf(4.f * m, light * 0x1p-10f));
    dmax[k] = 0u;
}

template <int ORDER, bool FROZEN, int GATHER, class Reg>
cudaError_t launch_t(pic_ctx *c, int si, const ExtDev &ext, Reg reg, int R3)
{
    const Species &s = c->sp[si];
    TileDev t = tile_dev(c, s);
    const size_t smem = (size_t)(FROZEN ? 0 : 6) * R3 * sizeof(float) + (size_t)3 * R3 * 2 * sizeof(int) +
                        (size_t)kQueue * 8 * sizeof(float);
    auto kern = k_push<ORDER, FROZEN, Reg, GATHER>;
    // attribute and occupancy once per kernel and region size (nothing but launches is then issued
    // while a step sequence is captured into a CUDA graph).  The cache is shared by every context
    // of the process: host threads driving contexts at once take it under a lock, and the shared-
    // memory attribute only grows, so a launch issued after the lock is released never meets a
    // smaller limit set by another thread.
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static size_t attr_max[kMaxDevices] = {};
    static size_t occ_smem = 0;
    static int occ_dev = -1, occ_per_sm = 0;
    cudaError_t e = cudaSuccess;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        const int dv = c->dev.device;
        if (dv < 0 || dv >= kMaxDevices) return cudaErrorInvalidDevice;
        if (attr_max[dv] < smem) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_max[dv] = smem;
        }
        if (occ_smem != smem || occ_dev != dv) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_per_sm, kern, kPushThreads, smem);
            if (e != cudaSuccess) return e;
            occ_smem = smem;
            occ_dev = dv;
        }
        per_sm = occ_per_sm;
    }
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    FieldsDev f{c->E, c->B, c->J};
    kern<<<c->num_sms * per_sm, kPushThreads, smem, c->stream>>>(species_dev(c, s), grid_dev(c), t, f, ext,
                                                                   c->work + si, c->work + kMaxSpecies + si, c->err,
                                                                   reg);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    float light[3];
    for (int d = 0; d < 3; d++) light[d] = (float)std::min(1.0, c->dt / c->d[d]);
    k_dlim_update<<<1, 32, 0, c->stream>>>(s.dlim, s.dmax, light[0], light[1], light[2]);
    c->kernels += 2;
    return cudaGetLastError();
}

// Compile-time region for the default tile (8^3 cells, drift margin 1); any other tuning uses
// the runtime-sized region.
inline bool default_region(const pic_ctx *c)
{
    return c->T[0] == 8 && c->T[1] == 8 && c->T[2] == 8 && c->M == 1;
}

// One kernel variant: shape order, frozen or mobile species, compile-time (FIXED) or runtime
// region, gather scheme (mobile species).  The second-order variants each sit in a translation
// unit of their own, so that the build compiles them in parallel.
template <int ORDER, bool FROZEN, bool FIXED, int GATHER = 0>
cudaError_t launch_variant(pic_ctx *c, int si, const ExtDev &ext)
{
    if constexpr (FIXED) {
        constexpr int R = 8 + 2 * 1 + (ORDER == 1 ? 3 : 5);
        RegFix<R, R, R> reg;
        constexpr int R3 = plane_pitch(R, R) * R;
        return launch_t<ORDER, FROZEN, GATHER>(c, si, ext, reg, R3);
    } else {
        const TileDev t = tile_dev(c, c->sp[si]);
        const int P2 = plane_pitch(t.R[0], t.R[1]);
        RegDyn reg{t.R[0], t.R[1], P2, P2 * t.R[2]};
        return launch_t<ORDER, FROZEN, GATHER>(c, si, ext, reg, reg.R3);
    }
}

template <int ORDER>
cudaError_t launch_order(pic_ctx *c, int si, const ExtDev &ext)
{
    const bool fr = c->sp[si].frozen != 0;
    const bool ec = c->gather == PIC_GATHER_ENERGY;
    if (default_region(c)) {
        if (fr) return launch_variant<ORDER, true, true>(c, si, ext);
        return ec ? launch_variant<ORDER, false, true, 1>(c, si, ext) : launch_variant<ORDER, false, true>(c, si, ext);
    }
    if (fr) return launch_variant<ORDER, true, false>(c, si, ext);
    return ec ? launch_variant<ORDER, false, false, 1>(c, si, ext) : launch_variant<ORDER, false, false>(c, si, ext);
}

}  // namespace push
}  // namespace gbpic
