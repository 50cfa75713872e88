// Lab-frame reconstruction at one lab time (Sec. "Understanding the RRF", Eq. DT): the particles of
// one RRF instant sit at different lab times (the time skew), so a lab snapshot at lab time T is
// assembled particle by particle as the RRF steps pass through T.  During step n a particle
// moves on a straight RRF segment from x^n (at t'_n) to x^{n+1} (at t'_n + dt) with momentum
// u^{n+1/2}; its lab time t = gamma_R (t' + beta_R z') grows along the segment.  When the step's
// lab-time interval [t_a, t_b) contains T, the event on the segment at lab time T is transformed
// to the lab (x, y unchanged, z = gamma_R (z' + beta_R t')), with the lab momentum of u^{n+1/2}
// (u_z = gamma_R (u'_z + beta_R gamma')), and recorded in FP64 under the particle's id.
#include "gbpic_internal.cuh"

#include <vector>

namespace gbpic {
namespace {

struct SnapP {
    CellCode cc;
    double d[3];
    float dt_over_d[3];
    double dt, tp, shifts, gR, bR, T;
    long long n_ids;
};

// RRF grid position (cells) of the particle after the push and its displacement of the step
// (the particle kernel's FP32 expression), both as doubles; z' absolute counts window shifts.
__device__ __forceinline__ void step_segment(const SnapP &p, float4 P, float4 Mo, double x1[3], double dx[3])
{
    const int cell = __float_as_int(P.w);
    x1[0] = (double)p.cc.i(cell) + (double)P.x;
    x1[1] = (double)p.cc.j(cell) + (double)P.y;
    x1[2] = (double)p.cc.k(cell) + (double)P.z + p.shifts;
    const float ig = rsqrtf(1.f + Mo.x * Mo.x + Mo.y * Mo.y + Mo.z * Mo.z);
    dx[0] = (double)(Mo.x * ig * p.dt_over_d[0]);
    dx[1] = (double)(Mo.y * ig * p.dt_over_d[1]);
    dx[2] = (double)(Mo.z * ig * p.dt_over_d[2]);
}

// Arming: a particle already at or past lab time T cannot be reconstructed (state 2: missed).
__global__ void k_snap_arm(SpeciesDev sp, SnapP p, unsigned char *state)
{
    const int n = sp.count[0];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const float4 P = sp.pos[q];
        const int cell = __float_as_int(P.w);
        if (cell < 0) continue;
        const int id = sp.id[q];
        if (id < 0 || id >= p.n_ids) continue;
        const double z = ((double)p.cc.k(cell) + (double)P.z + p.shifts) * p.d[2];
        if (p.gR * (p.tp + p.bR * z) >= p.T) state[id] = 2;
    }
}

__global__ void k_snap_record(SpeciesDev sp, SnapP p, double *rec, unsigned char *state)
{
    const int n = sp.count[0];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const float4 P = sp.pos[q];
        if (__float_as_int(P.w) < 0) continue;
        const int id = sp.id[q];
        if (id < 0 || id >= p.n_ids || state[id] != 0) continue;
        const float4 Mo = sp.mom[q];
        double x1[3], dx[3];
        step_segment(p, P, Mo, x1, dx);
        const double z1 = x1[2] * p.d[2], z0 = (x1[2] - dx[2]) * p.d[2];
        const double ta = p.gR * (p.tp + p.bR * z0), tb = p.gR * (p.tp + p.dt + p.bR * z1);
        if (!(ta < p.T && p.T <= tb)) continue;
        const double a = (p.T - ta) / (tb - ta);
        const double xp = (x1[0] - dx[0] + a * dx[0]) * p.d[0];
        const double yp = (x1[1] - dx[1] + a * dx[1]) * p.d[1];
        const double zp = z0 + a * (z1 - z0);
        const double tp = p.tp + a * p.dt;
        const double u[3] = {Mo.x, Mo.y, Mo.z};
        const double gp = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double *r = rec + 7 * (long long)id;
        r[0] = xp;
        r[1] = yp;
        r[2] = p.gR * (zp + p.bR * tp);
        r[3] = u[0];
        r[4] = u[1];
        r[5] = p.gR * (u[2] + p.bR * gp);
        r[6] = Mo.w;
        state[id] = 1;
    }
}

constexpr int kSnapK = 10;

// FP64 statistics of the recorded particles, in three passes (sums; means; central moments and
// bunching), the definitions of the species moments.
__global__ void k_snap_moments(const double *rec, const unsigned char *state, long long n, int pass,
                               const double *mean, double k, double mass, double *partial)
{
    double acc[kSnapK];
#pragma unroll
    for (int j = 0; j < kSnapK; j++) acc[j] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (state[i] != 1) continue;
        const double *r = rec + 7 * i;
        const double w = r[6];
        const double g = sqrt(1.0 + r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
        if (pass == 0) {
            acc[0] += w;
            acc[2] += 1.0;
        } else if (pass == 1) {
            for (int j = 0; j < 6; j++) acc[j] += w * r[j];
            acc[6] += w * g;
            acc[7] += w * mass * (g - 1.0);
        } else {
            const double dx = r[0] - mean[0], dy = r[1] - mean[1], dz = r[2] - mean[2];
            const double dux = r[3] - mean[3], duy = r[4] - mean[4], dg = g - mean[6];
            acc[0] += w * dx * dx; acc[1] += w * dy * dy; acc[2] += w * dz * dz;
            acc[3] += w * dux * dux; acc[4] += w * duy * duy;
            acc[5] += w * dx * dux; acc[6] += w * dy * duy;
            acc[7] += w * dg * dg;
            double sn, cs;
            sincos(k * dz, &sn, &cs);
            acc[8] += w * cs;
            acc[9] -= w * sn;
        }
    }
    __shared__ double ws[kSnapK][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kSnapK; j++) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) ws[j][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSnapK) {
        double v = 0.0;
        for (int k2 = 0; k2 < (int)(blockDim.x >> 5); k2++) v += ws[threadIdx.x][k2];
        partial[blockIdx.x * kSnapK + threadIdx.x] = v;
    }
}

SnapP snap_params(const pic_ctx *c)
{
    SnapP p{};
    p.cc = c->cc;
    for (int d = 0; d < 3; d++) {
        p.d[d] = c->d[d];
        p.dt_over_d[d] = (float)(c->dt / c->d[d]);
    }
    p.dt = c->dt;
    p.tp = (double)c->step * c->dt;
    p.shifts = (double)c->shifts;
    p.gR = c->gR;
    p.bR = c->bR;
    p.T = c->snap_T;
    p.n_ids = c->snap_n;
    return p;
}

}  // namespace

cudaError_t launch_snap_arm(pic_ctx *c)
{
    const Species &s = c->sp[c->snap_sp];
    k_snap_arm<<<c->num_sms * 4, 256, 0, c->stream>>>(species_dev(c, s), snap_params(c), c->snap_state);
    c->kernels++;
    return cudaGetLastError();
}

cudaError_t launch_snap_record(pic_ctx *c)
{
    const Species &s = c->sp[c->snap_sp];
    k_snap_record<<<c->num_sms * 4, 256, 0, c->stream>>>(species_dev(c, s), snap_params(c), c->snap, c->snap_state);
    c->kernels++;
    return cudaGetLastError();
}

// Moments of the recorded snapshot in the layout of pic_moments (mean_t: the snapshot's lab time).
cudaError_t launch_snap_moments(pic_ctx *c, double k, double *out)
{
    const int blocks = 512;
    std::vector<double> part((size_t)blocks * kSnapK);
    double sums[3][kSnapK];
    double mean[7] = {0, 0, 0, 0, 0, 0, 0};
    double *dmean = c->red + (size_t)blocks * kSnapK;   // after the partials
    const double mass = c->sp[c->snap_sp].m;
    for (int pass = 0; pass < 3; pass++) {
        cudaError_t e = cudaMemcpyAsync(dmean, mean, sizeof(mean), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return e;
        k_snap_moments<<<blocks, 256, 0, c->stream>>>(c->snap, c->snap_state, c->snap_n, pass, dmean, k, mass, c->red);
        c->kernels++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        e = cudaMemcpyAsync(part.data(), c->red, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
        for (int j = 0; j < kSnapK; j++) {
            double v = 0.0;
            for (int b = 0; b < blocks; b++) v += part[(size_t)b * kSnapK + j];
            sums[pass][j] = v;
        }
        if (pass == 1 && sums[0][0] > 0)
            for (int j = 0; j < 7; j++) mean[j] = sums[1][j] / sums[0][0];
    }
    const double sw = sums[0][0];
    for (int j = 0; j < 20; j++) out[j] = 0.0;
    out[0] = sums[0][2];
    out[1] = sw;
    out[2] = c->sp[c->snap_sp].q * sw;
    if (sw > 0) {
        const double *cs = sums[2];
        for (int d = 0; d < 3; d++) {
            out[3 + d] = mean[d];
            out[6 + d] = sqrt(cs[d] / sw);
            out[9 + d] = mean[3 + d];
        }
        out[12] = mean[6];
        out[13] = sqrt(cs[7] / sw) / mean[6];
        const double ex = (cs[0] / sw) * (cs[3] / sw) - (cs[5] / sw) * (cs[5] / sw);
        const double ey = (cs[1] / sw) * (cs[4] / sw) - (cs[6] / sw) * (cs[6] / sw);
        out[14] = sqrt(ex > 0 ? ex : 0.0);
        out[15] = sqrt(ey > 0 ? ey : 0.0);
        out[16] = sqrt(cs[8] * cs[8] + cs[9] * cs[9]) / sw;
        out[17] = sums[1][7];
    }
    out[18] = c->snap_T;
    return cudaSuccess;
}

}  // namespace gbpic
