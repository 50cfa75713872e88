// The dispatcher over the particle kernel's variants (shape order, frozen or mobile, region
// shape; the second-order variants are compiled in k_push2_*.cu, the first-order ones in
// k_push1.cu) and the charge-density deposit used by pic_get_fields(RHO).
#include "push_impl.cuh"

namespace gbpic {

cudaError_t launch_push_order1(pic_ctx *c, int si, const ExtDev &ext);
cudaError_t launch_push2_mobile_fixed(pic_ctx *c, int si, const ExtDev &ext);
cudaError_t launch_push2_frozen_fixed(pic_ctx *c, int si, const ExtDev &ext);
cudaError_t launch_push2_mobile_dyn(pic_ctx *c, int si, const ExtDev &ext);
cudaError_t launch_push2_frozen_dyn(pic_ctx *c, int si, const ExtDev &ext);
cudaError_t launch_push2_mobile_fixed_ec(pic_ctx *c, int si, const ExtDev &ext);
cudaError_t launch_push2_mobile_dyn_ec(pic_ctx *c, int si, const ExtDev &ext);

namespace {

// Charge density at the nodes: rho += q w S(node - x) / V for every live particle.
template <int ORDER>
__global__ void k_rho(SpeciesDev sp, GridDev g, float qv, float *rho)
{
    using S = push::Shape<ORDER>;
    const int n = sp.count[0];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 P = sp.pos[p];
        const int cell = __float_as_int(P.w);
        if (cell < 0) continue;
        const float w = sp.mom[p].w * qv;
        int c[3] = {g.cc.i(cell), g.cc.j(cell), g.cc.k(cell)};
        const int zb = zblock(c[2], g.nzr);
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
                    for (int d = 0; d < 2; d++) {
                        if (q[d] < 0 || q[d] >= g.n[d]) {
                            if (g.periodic[d]) q[d] = pwrap(q[d], g.n[d]);
                            else ok = false;
                        }
                    }
                    if (q[2] < zb || q[2] >= zb + g.nzr) {
                        if (g.periodic[2]) q[2] = zb + pwrap(q[2] - zb, g.nzr);
                        else ok = false;
                    }
                    if (ok)
                        atomicAdd(rho + ((long long)q[2] * g.n[1] + q[1]) * g.n[0] + q[0],
                                  w * wu[0][i] * wu[1][j] * wu[2][k]);
                }
    }
}

// Largest displacement per component the stored momenta give in one step, |u_c| dt / (gamma d_c).
__global__ void k_dmax_measure(SpeciesDev sp, float tx, float ty, float tz)
{
    unsigned m[3] = {0u, 0u, 0u};
    const int n = sp.count[0];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        if (__float_as_int(sp.pos[p].w) < 0) continue;
        const float4 u = sp.mom[p];
        const float ig = rsqrtf(1.f + u.x * u.x + u.y * u.y + u.z * u.z);
        m[0] = max(m[0], __float_as_uint(fabsf(u.x) * ig * tx));
        m[1] = max(m[1], __float_as_uint(fabsf(u.y) * ig * ty));
        m[2] = max(m[2], __float_as_uint(fabsf(u.z) * ig * tz));
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const unsigned r = __reduce_max_sync(0xffffffffu, m[k]);
        if ((threadIdx.x & 31) == 0 && r) atomicMax(sp.dmax + k, r);
    }
}

}  // namespace

// Sets the displacement bound of species si from its current momenta (after a load or an
// injection): four times the largest displacement they give, as after a step.
cudaError_t launch_dlim_from_momenta(pic_ctx *c, int si)
{
    const Species &s = c->sp[si];
    if (s.lattice || !s.dlim) return cudaSuccess;
    float light[3];
    for (int d = 0; d < 3; d++) light[d] = (float)std::min(1.0, c->dt / c->d[d]);
    k_dmax_measure<<<c->num_sms * 4, 256, 0, c->stream>>>(species_dev(c, s), (float)(c->dt / c->d[0]),
                                                          (float)(c->dt / c->d[1]), (float)(c->dt / c->d[2]));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    push::k_dlim_update<<<1, 32, 0, c->stream>>>(s.dlim, s.dmax, light[0], light[1], light[2]);
    c->kernels += 2;
    return cudaGetLastError();
}

cudaError_t launch_push(pic_ctx *c, int si, const ExtDev &ext)
{
    if (c->order == 1) return launch_push_order1(c, si, ext);
    const bool fr = c->sp[si].frozen != 0;
    const bool ec = c->gather == PIC_GATHER_ENERGY;
    if (push::default_region(c)) {
        if (fr) return launch_push2_frozen_fixed(c, si, ext);
        return ec ? launch_push2_mobile_fixed_ec(c, si, ext) : launch_push2_mobile_fixed(c, si, ext);
    }
    if (fr) return launch_push2_frozen_dyn(c, si, ext);
    return ec ? launch_push2_mobile_dyn_ec(c, si, ext) : launch_push2_mobile_dyn(c, si, ext);
}

// Adds the charge density of species s to rho.
cudaError_t launch_rho(pic_ctx *c, const Species &s, float *rho)
{
    const float V = (float)(c->d[0] * c->d[1] * c->d[2]);
    const float qv = (float)(s.q / V);
    if (c->order == 1) k_rho<1><<<c->num_sms * 8, 256, 0, c->stream>>>(species_dev(c, s), grid_dev(c), qv, rho);
    else k_rho<2><<<c->num_sms * 8, 256, 0, c->stream>>>(species_dev(c, s), grid_dev(c), qv, rho);
    c->kernels++;
    return cudaGetLastError();
}

}  // namespace gbpic
