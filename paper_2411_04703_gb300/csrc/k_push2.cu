// Second-order (TSC) instantiation of the fused particle kernel (see push_impl.cuh), the
// dispatcher over shape orders, and the charge-density deposit used by pic_get_fields(RHO).
#include "push_impl.cuh"

namespace gbpic {

cudaError_t launch_push_order1(pic_ctx *c, int si, const ExtDev &ext);

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
    return c->order == 1 ? launch_push_order1(c, si, ext) : push::launch_order<2>(c, si, ext);
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
