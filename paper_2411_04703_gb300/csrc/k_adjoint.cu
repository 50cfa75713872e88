// Hand-written discrete adjoint of one PIC step (first-order shape, periodic grid), used by
// pic_backward to differentiate a beam diagnostic with respect to the undulator K and the plasma
// density profile.
//
// Forward step n (Sec. "Relativistic booster frame": leap-frog push, current weighting, Maxwell):
//   F   = G(x^n; E^n, B^n) + F_ext(x^n, t_n; K)          gather at the Yee points + undulator
//   u+  = Boris(u^{n-1/2}, F)                              u^{n+1/2}
//   x^{n+1} = x^n + d(u+),  d_c = u+_c dt / (gamma+ d_c)
//   J   = D(x^n, x^{n+1}; w) + J_ions(w_planes)            Esirkepov + frozen lattice ions
//   (E, B)^{n+1} = M(E^n, B^n, J)                          Yee, B in two half steps
// The adjoint runs the steps backwards: M^T gives the adjoint current lambda_J and updates the
// field adjoints; per particle the forward step is recomputed in registers from the recorded
// x^n, u^{n-1/2}, E^n, B^n and reversed through deposit, move, Boris and gather (the gather's
// transpose scatters into the field adjoints, the deposit's transpose gathers lambda_J).  K
// enters through F_ext, the profile through the weights of the plasma electrons and ions.
// Everything here is FP32 except the parameter accumulators (FP64); the shape derivatives are
// those of the mathematical CIC shape (the window of a step is fixed by the forward move).
#include "gbpic_internal.cuh"

#include <algorithm>
#include <cmath>

namespace gbpic {
namespace {

constexpr int kAdjThreads = 256;

__device__ __forceinline__ int wrapi(int i, int n) { return pwrap(i, n); }

__device__ __forceinline__ long long nidx(const GridDev &g, int i, int j, int k)
{
    return ((long long)wrapi(k, g.n[2]) * g.n[1] + wrapi(j, g.n[1])) * g.n[0] + wrapi(i, g.n[0]);
}

// CIC shape S(t) = max(0, 1 - |t|) and its derivative.
__device__ __forceinline__ float S1(float t) { return fmaxf(0.f, 1.f - fabsf(t)); }
__device__ __forceinline__ float dS1(float t) { return fabsf(t) < 1.f ? (t > 0.f ? -1.f : 1.f) : 0.f; }

// Gather weights of the first-order shape at the integer nodes (unstaggered) and at the
// half-integer nodes (staggered), with their derivatives along the offset.
__device__ __forceinline__ void w_unst(float o, int &s, float w[2], float dw[2])
{
    s = 0;
    w[0] = 1.f - o; w[1] = o;
    dw[0] = -1.f; dw[1] = 1.f;
}
__device__ __forceinline__ void w_stag(float o, int &s, float w[2], float dw[2])
{
    const bool hi = o >= 0.5f;
    const float f = hi ? o - 0.5f : o + 0.5f;
    s = hi ? 0 : -1;
    w[0] = 1.f - f; w[1] = f;
    dw[0] = -1.f; dw[1] = 1.f;
}

// ------------------------------------------------------------------ field adjoint (M^T)
// lamE -= h curl_B(lamB)   (backward differences; the transpose of the forward-difference curl)
__global__ void k_adj_e(float *lE, const float *lB, GridDev g, float h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= g.n[0]) return;
    const long long N = g.ncell, ix = nidx(g, i, j, k);
    const float *Bx = lB, *By = lB + N, *Bz = lB + 2 * N;
    const float idx = 1.f / g.d[0], idy = 1.f / g.d[1], idz = 1.f / g.d[2];
    const float cx = (Bz[ix] - Bz[nidx(g, i, j - 1, k)]) * idy - (By[ix] - By[nidx(g, i, j, k - 1)]) * idz;
    const float cy = (Bx[ix] - Bx[nidx(g, i, j, k - 1)]) * idz - (Bz[ix] - Bz[nidx(g, i - 1, j, k)]) * idx;
    const float cz = (By[ix] - By[nidx(g, i - 1, j, k)]) * idx - (Bx[ix] - Bx[nidx(g, i, j - 1, k)]) * idy;
    lE[ix] -= h * cx;
    lE[N + ix] -= h * cy;
    lE[2 * N + ix] -= h * cz;
}

// lamB += dt curl_E(lamE) (forward differences); lamJ = -dt lamE when lJ is given
__global__ void k_adj_b(float *lB, const float *lE, float *lJ, GridDev g, float dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= g.n[0]) return;
    const long long N = g.ncell, ix = nidx(g, i, j, k);
    const float *Ex = lE, *Ey = lE + N, *Ez = lE + 2 * N;
    const float idx = 1.f / g.d[0], idy = 1.f / g.d[1], idz = 1.f / g.d[2];
    const float cx = (Ez[nidx(g, i, j + 1, k)] - Ez[ix]) * idy - (Ey[nidx(g, i, j, k + 1)] - Ey[ix]) * idz;
    const float cy = (Ex[nidx(g, i, j, k + 1)] - Ex[ix]) * idz - (Ez[nidx(g, i + 1, j, k)] - Ez[ix]) * idx;
    const float cz = (Ey[nidx(g, i + 1, j, k)] - Ey[ix]) * idx - (Ex[nidx(g, i, j + 1, k)] - Ex[ix]) * idy;
    lB[ix] += dt * cx;
    lB[N + ix] += dt * cy;
    lB[2 * N + ix] += dt * cz;
}

__global__ void k_adj_j(float *lJ, const float *lE, long long n3, float dt)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3; q += (long long)gridDim.x * blockDim.x)
        lJ[q] = -dt * lE[q];
}

// ------------------------------------------------------------------ particle adjoint
struct AdjP {
    GridDev g;
    SpeciesDev sp;           // the recorded particles of step n (pos, mom, id; count)
    const float *E, *B;      // recorded E^n, B^n
    const float *lJ;         // adjoint current of step n
    float *lE, *lB;          // field adjoints (gather transpose adds here)
    float4 *lx, *lu;         // per slot: adjoint of x^{n+1} (in) / x^n (out), of u^{n+1/2} (in) / u^{n-1/2} (out)
    double *lw;              // per particle id: adjoint of the weight (accumulated over steps)
    double *lK;              // adjoint of K (block partial sums)
    ExtDev ext;              // external field of step n (theta, amplitude)
    float K;                 // undulator strength (dF_ext/dK = F_ext / K)
    int n;
};

template <int N3> __device__ __forceinline__ float dot3(const float a[N3], const float b[N3])
{
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < N3; q++) s = fmaf(a[q], b[q], s);
    return s;
}

__device__ __forceinline__ void cross(const float a[3], const float b[3], float c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// PASS 0: the whole particle adjoint in one kernel.  PASS 1 and 2 split it around a per-record
// intermediate so that neither half keeps the other's values live (the single kernel spills):
// pass 1 recomputes the forward step and reverses the deposit and the move, leaving in lx the
// position adjoint gathered so far and in lu the adjoint of u^{n+1/2}; pass 2 recomputes the
// gather (with its derivatives) and Boris, reverses Boris and the gather, and writes the final
// adjoints of x^n and u^{n-1/2}.  Both passes do the same arithmetic as the single kernel.
template <int PASS>
__global__ void __launch_bounds__(kAdjThreads, 2) k_adj_particles(AdjP a)
{
    const GridDev &g = a.g;
    const unsigned lane = threadIdx.x & 31u;
    double kacc = 0.0;
    // consecutive threads take consecutive (cell-sorted) particles: coalesced record loads; the
    // scatters of a warp then often hit the same nodes, which measured cheaper than spreading the
    // lanes over the records (uncoalesced loads: 5.1 vs 3.7 ms per step on the 64x64x256 run).
    // Whole warps iterate together (the scatter below shuffles between lanes): a lane past the
    // end or on an empty slot computes a stand-in particle at cell 0 and neither scatters nor
    // stores.
    for (int base = blockIdx.x * blockDim.x; base < a.n; base += gridDim.x * blockDim.x) {
        const int p = base + (int)threadIdx.x;
        float4 P = p < a.n ? a.sp.pos[p] : make_float4(0.5f, 0.5f, 0.5f, __int_as_float(-1));
        const bool live = __float_as_int(P.w) >= 0;
        if (!live) P = make_float4(0.5f, 0.5f, 0.5f, __int_as_float(0));
        const int cell = __float_as_int(P.w);
        const float4 Mo = live ? a.sp.mom[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int c[3] = {g.cc.i(cell), g.cc.j(cell), g.cc.k(cell)};
        const float o[3] = {P.x, P.y, P.z};
        // wrapped node coordinates for the offsets -1 .. 2 the gather and deposit windows use,
        // pre-multiplied by the strides (a node index is then two additions); every index into
        // these tables below is a compile-time constant after unrolling, so they stay in registers
        int on[3][4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            on[0][q] = wrapi(c[0] + q - 1, g.n[0]);
            on[1][q] = wrapi(c[1] + q - 1, g.n[1]) * g.n[0];
            on[2][q] = wrapi(c[2] + q - 1, g.n[2]) * g.n[0] * g.n[1];
        }
        // ---- recompute the forward step: gather (+ external field), Boris, move
        float wu[3][2], ws[3][2], dwu[3][2], dws[3][2];
        int nu[3][2], ns[3][2];    // node offsets of the unstaggered / staggered gather windows
        int oct = 0;               // which staggered window each dim takes (with the cell: all 48 nodes)
#pragma unroll
        for (int d = 0; d < 3; d++) {
            int su, ss;
            w_unst(o[d], su, wu[d], dwu[d]);
            w_stag(o[d], ss, ws[d], dws[d]);
            oct |= (ss != 0) << d;
            nu[d][0] = on[d][1];
            nu[d][1] = on[d][2];
            ns[d][0] = ss ? on[d][0] : on[d][1];
            ns[d][1] = ss ? on[d][1] : on[d][2];
        }
        // component comp uses staggered weights along its own axis for E, along the other two for B
        float F[6], dF[6][3];
#pragma unroll
        for (int comp = 0; comp < 6; comp++) {
            const bool st0 = comp < 3 ? comp == 0 : comp != 3;
            const bool st1 = comp < 3 ? comp == 1 : comp != 4;
            const bool st2 = comp < 3 ? comp == 2 : comp != 5;
            const float *fld = comp < 3 ? a.E + comp * g.ncell : a.B + (comp - 3) * g.ncell;
            float v = 0.f, dv[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 2; k++)
#pragma unroll
                for (int j = 0; j < 2; j++)
#pragma unroll
                    for (int i = 0; i < 2; i++) {
                        const float wx = st0 ? ws[0][i] : wu[0][i], dx_ = st0 ? dws[0][i] : dwu[0][i];
                        const float wy = st1 ? ws[1][j] : wu[1][j], dy_ = st1 ? dws[1][j] : dwu[1][j];
                        const float wz = st2 ? ws[2][k] : wu[2][k], dz_ = st2 ? dws[2][k] : dwu[2][k];
                        const int ix = (st0 ? ns[0][i] : nu[0][i]) + (st1 ? ns[1][j] : nu[1][j]) + (st2 ? ns[2][k] : nu[2][k]);
                        const float f = __ldg(fld + ix);
                        v = fmaf(wx * wy * wz, f, v);
                        if constexpr (PASS != 1) {
                            dv[0] = fmaf(dx_ * wy * wz, f, dv[0]);
                            dv[1] = fmaf(wx * dy_ * wz, f, dv[1]);
                            dv[2] = fmaf(wx * wy * dz_, f, dv[2]);
                        }
                    }
            F[comp] = v;
#pragma unroll
            for (int d = 0; d < 3; d++) dF[comp][d] = dv[d];
        }
        float By_ext = 0.f, dBy_dz = 0.f;
        if (a.ext.type == PIC_EXT_PLANAR_UNDULATOR) {
            const float ph = a.ext.phase_tab[c[2]] + fmaf(a.ext.kdz, o[2], a.ext.theta);
            float sn, cs;
            sincosf(ph, &sn, &cs);
            By_ext = a.ext.B0g * cs;
            dBy_dz = -a.ext.B0g * sn * a.ext.kdz;
            F[4] += By_ext;
            F[0] -= a.ext.beta_R * By_ext;
        }
        const float h = a.sp.h_qm;
        const float E[3] = {F[0], F[1], F[2]}, B[3] = {F[3], F[4], F[5]};
        const float u0[3] = {Mo.x, Mo.y, Mo.z};
        float um[3];
        for (int d = 0; d < 3; d++) um[d] = fmaf(h, E[d], u0[d]);
        const float ig = rsqrtf(1.f + dot3<3>(um, um));
        float t[3];
        for (int d = 0; d < 3; d++) t[d] = h * B[d] * ig;
        const float s2 = 2.f / (1.f + dot3<3>(t, t));
        float umxt[3], up[3], sv[3], upxs[3], u1[3];
        cross(um, t, umxt);
        for (int d = 0; d < 3; d++) up[d] = um[d] + umxt[d];
        for (int d = 0; d < 3; d++) sv[d] = s2 * t[d];
        cross(up, sv, upxs);
        for (int d = 0; d < 3; d++) u1[d] = um[d] + upxs[d] + h * E[d];
        const float ig1 = rsqrtf(1.f + dot3<3>(u1, u1));
        float dd[3];
        for (int d = 0; d < 3; d++) dd[d] = u1[d] * ig1 * g.dt_over_d[d];
        float lo[3] = {0.f, 0.f, 0.f};
        float lu1[3];
        if constexpr (PASS == 2) {
            // pass 1's position adjoint so far and adjoint of u^{n+1/2}
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 LX = live ? a.lx[p] : z4, LU = live ? a.lu[p] : z4;
            lo[0] = LX.x; lo[1] = LX.y; lo[2] = LX.z;
            lu1[0] = LU.x; lu1[1] = LU.y; lu1[2] = LU.z;
        } else {
        // ---- adjoint of the deposit (general window of three nodes per dim)
        const float w = Mo.w;
        int st[3], wn[3][3];       // window start (-1 or 0) and the window's node offsets
        float S0[3][3], Sn[3][3], DS[3][3], A[3][3], Q[3][3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const int sh = (int)floorf(o[d] + dd[d]);
            st[d] = min(sh, 0);
#pragma unroll
            for (int q = 0; q < 3; q++) wn[d][q] = st[d] ? on[d][q] : on[d][q + 1];
            for (int q = 0; q < 3; q++) {
                S0[d][q] = S1(o[d] - (float)(st[d] + q));
                Sn[d][q] = S1(o[d] + dd[d] - (float)(st[d] + q));
                DS[d][q] = Sn[d][q] - S0[d][q];
                A[d][q] = S0[d][q] + 0.5f * DS[d][q];
                Q[d][q] = DS[d][q] * (1.f / 12.f);
            }
        }
        float lA[3][3] = {}, lQ[3][3] = {}, lDS[3][3] = {};
        float lw_step = 0.f;
#pragma unroll
        for (int comp = 0; comp < 3; comp++) {
            const int a1 = (comp + 1) % 3, a2 = (comp + 2) % 3;   // the two other dims (cyclic)
            const float fac = a.sp.cf[comp] * w;
            float pre[2];
            pre[0] = DS[comp][0];
            pre[1] = DS[comp][0] + DS[comp][1];
            float lP[2] = {0.f, 0.f};
#pragma unroll
            for (int q2 = 0; q2 < 3; q2++)
#pragma unroll
                for (int q1 = 0; q1 < 3; q1++) {
                    const float Y = fmaf(A[a1][q1], A[a2][q2], Q[a1][q1] * DS[a2][q2]);
                    float lY = 0.f;
#pragma unroll
                    for (int q0 = 0; q0 < 2; q0++) {
                        const int ix = wn[comp][q0] + wn[a1][q1] + wn[a2][q2];
                        const float lj = __ldg(a.lJ + comp * g.ncell + ix);
                        lP[q0] = fmaf(lj, Y, lP[q0]);
                        lY = fmaf(lj, fac * pre[q0], lY);
                    }
                    lA[a1][q1] = fmaf(lY, A[a2][q2], lA[a1][q1]);
                    lA[a2][q2] = fmaf(lY, A[a1][q1], lA[a2][q2]);
                    lQ[a1][q1] = fmaf(lY, DS[a2][q2], lQ[a1][q1]);
                    lDS[a2][q2] = fmaf(lY, Q[a1][q1], lDS[a2][q2]);
                }
            // J = fac * pre * Y: weight adjoint and the prefix's adjoint
            lw_step += a.sp.cf[comp] * (lP[0] * pre[0] + lP[1] * pre[1]);
            lDS[comp][0] += fac * (lP[0] + lP[1]);
            lDS[comp][1] += fac * lP[1];
        }
        // A = S0 + DS/2, Q = DS/12, DS = Sn - S0; S0 = S(o - m), Sn = S(o + d - m)
        float ld[3] = {0.f, 0.f, 0.f};
        for (int d = 0; d < 3; d++)
            for (int q = 0; q < 3; q++) {
                const float lds = lDS[d][q] + 0.5f * lA[d][q] + lQ[d][q] * (1.f / 12.f);
                const float lS0 = lA[d][q] - lds;
                const float lSn = lds;
                const float m = (float)(st[d] + q);
                lo[d] += lS0 * dS1(o[d] - m) + lSn * dS1(o[d] + dd[d] - m);
                ld[d] += lSn * dS1(o[d] + dd[d] - m);
            }
        // ---- adjoint of the move x^{n+1} = x^n + d(u+)
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 LX = live ? a.lx[p] : z4, LU = live ? a.lu[p] : z4;
        const float lx1[3] = {LX.x, LX.y, LX.z};
        for (int d = 0; d < 3; d++) {
            lo[d] += lx1[d];
            ld[d] += lx1[d];
        }
        lu1[0] = LU.x; lu1[1] = LU.y; lu1[2] = LU.z;
        {
            float sdot = 0.f;
            for (int d = 0; d < 3; d++) sdot += ld[d] * g.dt_over_d[d] * u1[d];
            const float ig3 = ig1 * ig1 * ig1;
            for (int d = 0; d < 3; d++) lu1[d] += ld[d] * g.dt_over_d[d] * ig1 - ig3 * u1[d] * sdot;
        }
        if (live) a.lw[a.sp.id[p]] += (double)lw_step;
        if constexpr (PASS == 1) {
            if (live) {
                a.lx[p] = make_float4(lo[0], lo[1], lo[2], 0.f);
                a.lu[p] = make_float4(lu1[0], lu1[1], lu1[2], 0.f);
            }
            continue;
        }
        }   // PASS != 2
        // ---- adjoint of Boris
        float lE[3], lB[3], lum[3], lup[3], lsv[3], lt[3];
        for (int d = 0; d < 3; d++) lE[d] = h * lu1[d];
        for (int d = 0; d < 3; d++) lum[d] = lu1[d];
        cross(sv, lu1, lup);                 // u1 += up x sv: lam_up = sv x lam
        cross(lu1, up, lsv);                 //                lam_sv = lam x up
        const float ls2 = dot3<3>(lsv, t);
        for (int d = 0; d < 3; d++) lt[d] = s2 * lsv[d] - s2 * s2 * t[d] * ls2;
        {
            float txl[3], lxu[3];
            cross(t, lup, txl);              // up = um + um x t: lam_um += lam_up + t x lam_up
            cross(lup, um, lxu);             //                  lam_t += lam_up x um
            for (int d = 0; d < 3; d++) {
                lum[d] += lup[d] + txl[d];
                lt[d] += lxu[d];
            }
        }
        for (int d = 0; d < 3; d++) lB[d] = h * ig * lt[d];
        const float lig = h * dot3<3>(B, lt);
        const float ig3m = ig * ig * ig;
        for (int d = 0; d < 3; d++) lum[d] += -ig3m * um[d] * lig;
        for (int d = 0; d < 3; d++) lE[d] += h * lum[d];
        const float lu0[3] = {lum[0], lum[1], lum[2]};
        // ---- adjoint of the gather and the external field
        const float lF[6] = {live ? lE[0] : 0.f, live ? lE[1] : 0.f, live ? lE[2] : 0.f,
                             live ? lB[0] : 0.f, live ? lB[1] : 0.f, live ? lB[2] : 0.f};
        // The 48 scatter targets follow from the cell and the staggered-window choice.  Where
        // all 32 lanes of the warp share both (the core of a dense beam, ~1000 particles per
        // cell, sorted by cell and octant), the warp sums the 48 values by a transpose
        // reduction: each exchange halves the values a lane holds (24, 12, 6, 3 for lane bits
        // 4..1; the last pair swaps all three), 48 shuffles in all; lane L ends with the totals
        // of value indices 3 (L >> 1) .. 3 (L >> 1) + 2 and issues one or two atomics.  Other
        // warps scatter their own values, 48 atomics per particle.
        const long long key = live ? (((long long)cell << 3) | oct) : -1ll - (long long)lane;
        const bool uniform = __all_sync(0xffffffffu, key == __shfl_sync(0xffffffffu, key, 0));
#pragma unroll
        for (int comp = 0; comp < 6; comp++)
#pragma unroll
            for (int d = 0; d < 3; d++) lo[d] = fmaf(lF[comp], dF[comp][d], lo[d]);
        if (uniform) {
            // value index vi = comp * 8 + k * 4 + j * 2 + i: its weight, then its node
            auto val = [&](int vi) {
                const int comp = vi >> 3, i = vi & 1, j = (vi >> 1) & 1, k = (vi >> 2) & 1;
                const bool st0 = comp < 3 ? comp == 0 : comp != 3;
                const bool st1 = comp < 3 ? comp == 1 : comp != 4;
                const bool st2 = comp < 3 ? comp == 2 : comp != 5;
                const float wx = st0 ? ws[0][i] : wu[0][i];
                const float wy = st1 ? ws[1][j] : wu[1][j];
                const float wz = st2 ? ws[2][k] : wu[2][k];
                return wx * wy * wz * lF[comp];
            };
            float h24[24], h12[12], h6[6], h3[3];
            const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u, b1 = lane & 2u;
#pragma unroll
            for (int q = 0; q < 24; q++) {
                const float lo_ = val(q), hi_ = val(24 + q);
                h24[q] = (b4 ? hi_ : lo_) + __shfl_xor_sync(0xffffffffu, b4 ? lo_ : hi_, 16);
            }
#pragma unroll
            for (int q = 0; q < 12; q++)
                h12[q] = (b3 ? h24[12 + q] : h24[q]) + __shfl_xor_sync(0xffffffffu, b3 ? h24[q] : h24[12 + q], 8);
#pragma unroll
            for (int q = 0; q < 6; q++)
                h6[q] = (b2 ? h12[6 + q] : h12[q]) + __shfl_xor_sync(0xffffffffu, b2 ? h12[q] : h12[6 + q], 4);
#pragma unroll
            for (int q = 0; q < 3; q++)
                h3[q] = (b1 ? h6[3 + q] : h6[q]) + __shfl_xor_sync(0xffffffffu, b1 ? h6[q] : h6[3 + q], 2);
#pragma unroll
            for (int q = 0; q < 3; q++) h3[q] += __shfl_xor_sync(0xffffffffu, h3[q], 1);
            const int vbase = 3 * (int)(lane >> 1);
#pragma unroll
            for (int q = 0; q < 3; q++) {
                if ((q < 2) == ((lane & 1u) == 0u)) {
                    const int vi = vbase + q;
                    const int comp = vi >> 3;
                    const int qq[3] = {vi & 1, (vi >> 1) & 1, (vi >> 2) & 1};
                    int ix = 0;
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        const bool st = comp < 3 ? comp == d : comp - 3 != d;
                        const int x = wrapi(c[d] + qq[d] - ((st && ((oct >> d) & 1)) ? 1 : 0), g.n[d]);
                        ix += d == 0 ? x : (d == 1 ? x * g.n[0] : x * g.n[0] * g.n[1]);
                    }
                    float *lf = comp < 3 ? a.lE + comp * g.ncell : a.lB + (comp - 3) * g.ncell;
                    atomicAdd(lf + ix, h3[q]);
                }
            }
        } else {
#pragma unroll
            for (int comp = 0; comp < 6; comp++) {
                const bool st0 = comp < 3 ? comp == 0 : comp != 3;
                const bool st1 = comp < 3 ? comp == 1 : comp != 4;
                const bool st2 = comp < 3 ? comp == 2 : comp != 5;
                float *lf = comp < 3 ? a.lE + comp * g.ncell : a.lB + (comp - 3) * g.ncell;
                if (lF[comp] != 0.f)
#pragma unroll
                    for (int k = 0; k < 2; k++)
#pragma unroll
                        for (int j = 0; j < 2; j++)
#pragma unroll
                            for (int i = 0; i < 2; i++) {
                                const float wx = st0 ? ws[0][i] : wu[0][i];
                                const float wy = st1 ? ws[1][j] : wu[1][j];
                                const float wz = st2 ? ws[2][k] : wu[2][k];
                                const int ix = (st0 ? ns[0][i] : nu[0][i]) + (st1 ? ns[1][j] : nu[1][j]) + (st2 ? ns[2][k] : nu[2][k]);
                                atomicAdd(lf + ix, wx * wy * wz * lF[comp]);
                            }
            }
        }
        if (a.ext.type == PIC_EXT_PLANAR_UNDULATOR) {
            const float lBy = lF[4] - a.ext.beta_R * lF[0];
            lo[2] = fmaf(lBy, dBy_dz, lo[2]);
            if (live && a.K != 0.f) kacc += (double)lBy * (double)By_ext / (double)a.K;
        }
        if (live) {
            a.lx[p] = make_float4(lo[0], lo[1], lo[2], 0.f);
            a.lu[p] = make_float4(lu0[0], lu0[1], lu0[2], 0.f);
        }
    }
    // adjoint of K: block reduction, one atomic per block
    for (int off = 16; off > 0; off >>= 1) kacc += __shfl_down_sync(0xffffffffu, kacc, off);
    __shared__ double ws_[kAdjThreads / 32];
    if ((threadIdx.x & 31) == 0) ws_[threadIdx.x >> 5] = kacc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kAdjThreads / 32; q++) s += ws_[q];
        atomicAdd(a.lK, s);
    }
}

// ------------------------------------------------------------------ frozen lattice ions
// J_z(i, j, k) = Tx(i) Ty(j) sum_m cf w_m prefix_m(k): lam_w_m += cf sum_k prefix_m(k) R(k) with
// R(k) = sum_ij Tx(i) Ty(j) lamJ_z(i, j, k).
__global__ void k_adj_ion_rows(const float *lJz, const float *tx, const float *ty, int nx, int ny, double *R)
{
    const int k = blockIdx.x;
    double s = 0.0;
    for (int q = threadIdx.x; q < nx * ny; q += blockDim.x) {
        const int i = q % nx, j = q / nx;
        s += (double)tx[i] * ty[j] * lJz[((long long)k * ny + j) * nx + i];
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += w[q];
        R[k] = t;
    }
}

__global__ void k_adj_ion_planes(const PlaneRec *planes, long long cap, const double *R, int nz, float uz, float dtdz,
                                 double cf, double *lw_plane)
{
    for (long long sidx = blockIdx.x * (long long)blockDim.x + threadIdx.x; sidx < cap; sidx += (long long)gridDim.x * blockDim.x) {
        const PlaneRec r = planes[sidx];
        if (r.kz < 0) continue;
        const float ig = rsqrtf(1.f + uz * uz);
        const float d = uz * ig * dtdz;
        const double z0 = (double)r.oz, z1 = z0 + (double)d;
        double run = 0.0, acc = 0.0;
        for (int nr = -1; nr <= 2; nr++) {
            run += shape_weight(1, (double)nr - z1) - shape_weight(1, (double)nr - z0);
            const int kk = ((r.kz + nr) % nz + nz) % nz;
            acc += run * R[kk];
        }
        lw_plane[sidx] += cf * acc;
    }
}

// ------------------------------------------------------------------ loss and bookkeeping
// L = |sum w e^{-i k z}| / sum w over the live particles (z in normalised RRF length):
// lam_z(p) = (a dA/dz_p + b dB/dz_p) / (|S| sum w), S = A + iB; lam_x in cells = lam_z dz.
__global__ void k_bunch_sums(SpeciesDev sp, GridDev g, double k, double shifts, double *out3)
{
    double a = 0.0, b = 0.0, sw = 0.0;
    const int n = sp.count[0];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 P = sp.pos[p];
        const int cell = __float_as_int(P.w);
        if (cell < 0) continue;
        const double w = sp.mom[p].w;
        const double z = ((double)g.cc.k(cell) + (double)P.z + shifts) * (double)g.d[2];
        double sn, cs;
        sincos(k * z, &sn, &cs);
        a += w * cs;
        b -= w * sn;
        sw += w;
    }
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
        sw += __shfl_down_sync(0xffffffffu, sw, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out3, a);
        atomicAdd(out3 + 1, b);
        atomicAdd(out3 + 2, sw);
    }
}

__global__ void k_bunch_seed(SpeciesDev sp, GridDev g, double k, double shifts, const double *sums, float4 *lx)
{
    const int n = sp.count[0];
    const double A = sums[0], B = sums[1], SW = sums[2];
    const double r = sqrt(A * A + B * B);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 P = sp.pos[p];
        const int cell = __float_as_int(P.w);
        float lz = 0.f;
        if (cell >= 0 && r > 0.0 && SW > 0.0) {
            const double w = sp.mom[p].w;
            const double z = ((double)g.cc.k(cell) + (double)P.z + shifts) * (double)g.d[2];
            double sn, cs;
            sincos(k * z, &sn, &cs);
            const double dl = (A * (-k * w * sn) + B * (-k * w * cs)) / (r * SW);
            lz = (float)(dl * (double)g.d[2]);
        }
        lx[p] = make_float4(0.f, 0.f, lz, 0.f);
    }
}

// Re-order the particle adjoints across a sort: the slot of id q before the sort is inv[q].
__global__ void k_adj_inverse(const int *id, int n, int *inv)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) inv[id[p]] = p;
}
__global__ void k_adj_remap(const int *id_after, int n, const int *inv_before, const float4 *lx, const float4 *lu,
                            float4 *lx_out, float4 *lu_out)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int q = inv_before[id_after[p]];
        lx_out[q] = lx[p];
        lu_out[q] = lu[p];
    }
}

// Profile gradient: dL/dn_j = sum over particles and ion planes of lam_w dw/dn_j, with
// w = gamma_R n_lab(z_lab) dV / ppc, n_lab piecewise linear through the nodes (hat functions),
// z_lab = gamma_R ((m + 1/2)/ppc_z) dz the lab position of lattice plane m (Eq. Nnormi).
__device__ __forceinline__ void hat_add(const double *zn, int np, double z, double v, double *grad)
{
    if (np <= 0 || z < zn[0] || z > zn[np - 1]) return;
    for (int q = 0; q + 1 < np; q++) {
        if (z <= zn[q + 1]) {
            const double hh = zn[q + 1] - zn[q];
            const double rr = hh > 0.0 ? (z - zn[q]) / hh : 0.0;
            atomicAdd(grad + q, v * (1.0 - rr));
            atomicAdd(grad + q + 1, v * rr);
            return;
        }
    }
}

__global__ void k_profile_grad(const double *lw, long long n_ids, long long per_plane, const double *lw_plane,
                               long long plane_cap, const double *zn, int np, double gR, double dz, int ppcz,
                               double wfac, double *grad)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n_ids + plane_cap;
         q += (long long)gridDim.x * blockDim.x) {
        long long m;
        double v;
        if (q < n_ids) {
            m = q / per_plane;          // electron id -> lattice plane
            v = lw[q];
        } else {
            m = q - n_ids;              // ion plane slot m (planes are never recycled in a periodic box)
            v = lw_plane[m];
        }
        if (v == 0.0) continue;
        const double zlab = gR * (((double)m + 0.5) / ppcz) * dz;
        hat_add(zn, np, zlab, v * wfac, grad);
    }
}

}  // namespace

// ---------------------------------------------------------------------------- launchers
cudaError_t adj_fields(pic_ctx *c, float *lE, float *lB, float *lJ)
{
    const GridDev g = grid_dev(c);
    const float h = (float)(0.5 * c->dt), dt = (float)c->dt;
    const dim3 grd((c->n[0] + 127) / 128, c->n[1], c->n[2]);
    k_adj_e<<<grd, 128, 0, c->stream>>>(lE, lB, g, h);
    k_adj_b<<<grd, 128, 0, c->stream>>>(lB, lE, nullptr, g, dt);
    k_adj_j<<<c->num_sms * 8, 256, 0, c->stream>>>(lJ, lE, 3 * c->ncell, dt);
    k_adj_e<<<grd, 128, 0, c->stream>>>(lE, lB, g, h);
    c->kernels += 4;
    return cudaGetLastError();
}

cudaError_t adj_particles(pic_ctx *c, const Species &rec, const float *E, const float *B, const float *lJ, float *lE,
                          float *lB, float4 *lx, float4 *lu, double *lw, double *lK, const ExtDev &ext, int n)
{
    if (n <= 0) return cudaSuccess;
    AdjP a;
    a.g = grid_dev(c);
    a.sp = species_dev(c, rec);
    a.E = E;
    a.B = B;
    a.lJ = lJ;
    a.lE = lE;
    a.lB = lB;
    a.lx = lx;
    a.lu = lu;
    a.lw = lw;
    a.lK = lK;
    a.ext = ext;
    a.K = (float)c->K;
    a.n = n;
    const int blocks = std::min((n + kAdjThreads - 1) / kAdjThreads, c->num_sms * 8);
    // two passes around the per-record intermediate in lx, lu (see k_adj_particles)
    k_adj_particles<1><<<blocks, kAdjThreads, 0, c->stream>>>(a);
    k_adj_particles<2><<<blocks, kAdjThreads, 0, c->stream>>>(a);
    c->kernels += 2;
    return cudaGetLastError();
}

cudaError_t adj_ions(pic_ctx *c, const Species &s, const PlaneRec *planes, const float *lJ, double *R, double *lw_plane)
{
    k_adj_ion_rows<<<c->n[2], 256, 0, c->stream>>>(lJ + 2 * c->ncell, s.tx, s.ty, c->n[0], c->n[1], R);
    const float uz = (float)(-std::sqrt(c->gR * c->gR - 1.0));
    const double cf = (double)species_dev(c, s).cf[2];
    const int blocks = (int)std::max<long long>(1, std::min<long long>((s.plane_cap + 255) / 256, (long long)c->num_sms));
    k_adj_ion_planes<<<blocks, 256, 0, c->stream>>>(planes, s.plane_cap, R, c->n[2], uz, (float)(c->dt / c->d[2]), cf,
                                                    lw_plane);
    c->kernels += 2;
    return cudaGetLastError();
}

cudaError_t adj_bunch_seed(pic_ctx *c, const Species &s, double k, double *sums_dev, double *host3, float4 *lx)
{
    cudaError_t e = cudaMemsetAsync(sums_dev, 0, 3 * sizeof(double), c->stream);
    if (e != cudaSuccess) return e;
    const GridDev g = grid_dev(c);
    k_bunch_sums<<<c->num_sms * 4, 256, 0, c->stream>>>(species_dev(c, s), g, k, (double)c->shifts, sums_dev);
    k_bunch_seed<<<c->num_sms * 4, 256, 0, c->stream>>>(species_dev(c, s), g, k, (double)c->shifts, sums_dev, lx);
    c->kernels += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaMemcpyAsync(host3, sums_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

cudaError_t adj_remap(pic_ctx *c, const int *id_before, int n_before, const int *id_after, int n_after, int *inv,
                      const float4 *lx, const float4 *lu, float4 *lx_out, float4 *lu_out)
{
    cudaError_t e = cudaMemsetAsync(lx_out, 0, sizeof(float4) * std::max(n_before, 1), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(lu_out, 0, sizeof(float4) * std::max(n_before, 1), c->stream);
    if (e != cudaSuccess) return e;
    if (n_before > 0) {
        k_adj_inverse<<<std::min((n_before + 255) / 256, c->num_sms * 8), 256, 0, c->stream>>>(id_before, n_before, inv);
        c->kernels++;
    }
    if (n_after > 0) {
        k_adj_remap<<<std::min((n_after + 255) / 256, c->num_sms * 8), 256, 0, c->stream>>>(id_after, n_after, inv, lx,
                                                                                             lu, lx_out, lu_out);
        c->kernels++;
    }
    return cudaGetLastError();
}

cudaError_t adj_profile_grad(pic_ctx *c, const double *lw_e, long long n_ids, const double *lw_plane, double *grad)
{
    const Species &si = c->sp[c->sp_i];
    const long long per_plane = (long long)(c->xr[1] - c->xr[0]) * (c->xr[3] - c->xr[2]) * c->ppc[0] * c->ppc[1];
    const double wfac = c->gR * c->d[0] * c->d[1] * c->d[2] / ((double)c->ppc[0] * c->ppc[1] * c->ppc[2]);
    const long long tot = n_ids + si.plane_cap;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((tot + 255) / 256, (long long)c->num_sms * 8));
    k_profile_grad<<<blocks, 256, 0, c->stream>>>(lw_e, n_ids, per_plane, lw_plane, si.plane_cap, c->prof, c->nprof,
                                                  c->gR, c->d[2], c->ppc[2], wfac, grad);
    c->kernels++;
    return cudaGetLastError();
}

}  // namespace gbpic
