// The frozen plasma ions as a lattice species (Sec. 2: the cold plasma is at rest in the lab,
// so in the RRF every ion drifts with u' = (0, 0, -gamma_R beta_R) and is never pushed).
//
// The ions are injected as a lab-static lattice: plane m holds the same transverse lattice
// (ppc_x x ppc_y points in every cell of the transverse range), every ion of the plane has the
// same z offset, cell row and weight, and every ion moves by the same displacement d along z.
// The charge-conserving current of one such ion (Esirkepov, with d_x = d_y = 0) is
//     J_z(i, j, k + 1/2) = cf_z w S_x(i - x) S_y(j - y) sum_{k' <= k} [S_z(k' - z - d) - S_z(k' - z)],
// J_x = J_y = 0, so the current of all ions factors exactly as
//     J_z(i, j, k + 1/2) = Tx(i) Ty(j) Z(k),
// with Tx(i) = sum over the lattice's x points of S_x(i - x) (likewise Ty), fixed at injection,
// and Z(k) = sum over live planes of cf_z w_m times the prefix sum of the plane's shape change,
// one step's 1-D work.  A step of the species is one pass over the planes (move as the particle
// kernel moves a frozen particle, drop below the margin, accumulate Z in FP64) and one pass over
// the grid that writes J_z.  The particle records that diagnostics read are materialised from the
// planes on demand (k_init.cu).
#include "gbpic_internal.cuh"

#include <algorithm>
#include <cmath>

namespace gbpic {
namespace {

struct LatStepP {
    PlaneRec *planes;
    long long cap;
    double *zacc;
    int nz, nzr, mlo, mhi, periodic, order;
    float uz, dtdz;
    double cf;
};

__global__ void k_lattice_step(LatStepP p, int *err)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < p.cap; s += (long long)gridDim.x * blockDim.x) {
        PlaneRec r = p.planes[s];
        if (r.kz < 0) continue;
        // the move of a frozen particle with u = (0, 0, u_z), in the particle kernel's FP32 steps
        const float ig = rsqrtf(1.f + p.uz * p.uz);
        const float d = p.uz * ig * p.dtdz;
        const float x1 = r.oz + d;
        int sh = (int)floorf(x1);
        float o1 = x1 - (float)sh;
        if (o1 >= 1.f) { o1 = 0.f; sh += 1; }
        if (sh < -1 || sh > 1) {
            atomicOr(err, ERR_MOVE);
            r.kz = -1;
            p.planes[s] = r;
            continue;
        }
        int kn = r.kz + sh;
        bool alive = true;
        const int zb = zblock(r.kz, p.nzr);   // the plane's run (ensembles: z wraps inside it)
        if (p.periodic) kn = zwrap(kn, zb, p.nzr);
        else if (kn < p.mlo || kn > p.nz - 1 - p.mhi) alive = false;
        if (alive) {
            // prefix sum of the shape change over the window; positions relative to the old row
            const double z0 = (double)r.oz, z1 = z0 + (double)d;
            const double fw = p.cf * (double)r.w;
            double run = 0.0;
            for (int nr = -p.order; nr <= p.order + 1; nr++) {
                run += shape_weight(p.order, (double)nr - z1) - shape_weight(p.order, (double)nr - z0);
                if (run == 0.0) continue;
                int kk = r.kz + nr;
                if (p.periodic) kk = zwrap(kk, zb, p.nzr);
                if (kk < 0 || kk >= p.nz) { atomicOr(err, ERR_INDEX); continue; }
                atomicAdd(&p.zacc[kk], fw * run);
            }
        }
        r.oz = o1;
        r.kz = alive ? kn : -1;
        p.planes[s] = r;
    }
}

__global__ void k_lattice_jz(float *jz, const float *tx, const float *ty, const double *zacc, int nx, int ny)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    jz[((long long)k * ny + j) * nx + i] = tx[i] * ty[j] * (float)zacc[k];
}

__global__ void k_lattice_shift(PlaneRec *planes, long long cap, int mlo)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < cap; s += (long long)gridDim.x * blockDim.x) {
        const int kz = planes[s].kz;
        if (kz < 0) continue;
        planes[s].kz = kz - 1 < mlo ? -1 : kz - 1;
    }
}

}  // namespace

// One step of the lattice species: writes J_z of the whole grid (every other species adds to it
// afterwards), so it runs first in the step.
cudaError_t launch_lattice_step(pic_ctx *c, int si)
{
    const Species &s = c->sp[si];
    cudaError_t e = cudaMemsetAsync(s.zacc, 0, sizeof(double) * c->n[2], c->stream);
    if (e != cudaSuccess) return e;
    LatStepP p{};
    p.planes = s.planes;
    p.cap = s.plane_cap;
    p.zacc = s.zacc;
    p.nz = c->n[2];
    p.nzr = c->nzr;
    p.mlo = c->order == 1 ? 1 : 2;
    p.mhi = c->order == 1 ? 2 : 3;
    p.periodic = c->bc[2][0] == PIC_BC_PERIODIC;
    p.order = c->order;
    p.uz = (float)(-std::sqrt(c->gR * c->gR - 1.0));
    p.dtdz = (float)(c->dt / c->d[2]);
    p.cf = (double)species_dev(c, s).cf[2];
    const int blocks = (int)std::min<long long>((s.plane_cap + 255) / 256, (long long)c->num_sms);
    k_lattice_step<<<blocks, 256, 0, c->stream>>>(p, c->err);
    const dim3 g((c->n[0] + 127) / 128, c->n[1], c->n[2]);
    k_lattice_jz<<<g, 128, 0, c->stream>>>(c->J + 2 * c->ncell, s.tx, s.ty, s.zacc, c->n[0], c->n[1]);
    c->kernels += 2;
    return cudaGetLastError();
}

cudaError_t launch_lattice_shift(pic_ctx *c, int si)
{
    const Species &s = c->sp[si];
    const int blocks = (int)std::min<long long>((s.plane_cap + 255) / 256, (long long)c->num_sms);
    k_lattice_shift<<<blocks, 256, 0, c->stream>>>(s.planes, s.plane_cap, c->order == 1 ? 1 : 2);
    c->kernels++;
    return cudaGetLastError();
}

}  // namespace gbpic
