// Yee FDTD update of Maxwell's equations in the RRF (Eq. Max1-Max2 normalised: dE/dt =
// curl B - J, dB/dt = -curl E), with B split into two half steps so that E^n and B^n are
// co-timed at the particle gather, and a convolutional PML (kappa = 1, alpha = 0) in the
// absorbing slabs ("the fields are absorbed upon interaction with the boundaries").
// One thread per cell, x fastest; neighbours outside a non-periodic face read as zero.
#include "gbpic_internal.cuh"

namespace gbpic {
namespace {

// Neighbour value; zb: first row of the run that owns the updated cell (0 for a single run).
__device__ __forceinline__ float ld(const float *F, const GridDev &g, int i, int j, int k, int zb)
{
    if (i >= g.n[0]) { if (!g.periodic[0]) return 0.f; i -= g.n[0]; }
    if (i < 0) { if (!g.periodic[0]) return 0.f; i += g.n[0]; }
    if (j >= g.n[1]) { if (!g.periodic[1]) return 0.f; j -= g.n[1]; }
    if (j < 0) { if (!g.periodic[1]) return 0.f; j += g.n[1]; }
    if (k >= zb + g.nzr) { if (!g.periodic[2]) return 0.f; k -= g.nzr; }
    if (k < zb) { if (!g.periodic[2]) return 0.f; k += g.nzr; }
    return __ldg(F + ((long long)k * g.n[1] + j) * g.n[0] + i);
}

// psi = b psi + (b - 1) dF; returns dF + psi (the CPML-stretched derivative).
__device__ __forceinline__ float cpml(float *psi, long long ix, float b, float dF)
{
    if (b >= 1.f) return dF;
    const float p = fmaf(b, psi[ix], (b - 1.f) * dF);
    psi[ix] = p;
    return dF + p;
}

// B -= dtt curl E (half step).  B_x at (i, j+1/2, k+1/2), B_y at (i+1/2, j, k+1/2),
// B_z at (i+1/2, j+1/2, k): forward differences of E.
__global__ void k_fdtd_b(FieldsDev f, GridDev g, PmlDev pml, float dtt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int zb = zblock(k, g.nzr);
    const long long N = g.ncell;
    const long long ix = ((long long)k * g.n[1] + j) * g.n[0] + i;
    const float *Ex = f.E, *Ey = f.E + N, *Ez = f.E + 2 * N;
    const float ex = Ex[ix], ey = Ey[ix], ez = Ez[ix];
    const float idx = 1.f / g.d[0], idy = 1.f / g.d[1], idz = 1.f / g.d[2];
    float dEz_dy = (ld(Ez, g, i, j + 1, k, zb) - ez) * idy;
    float dEy_dz = (ld(Ey, g, i, j, k + 1, zb) - ey) * idz;
    float dEx_dz = (ld(Ex, g, i, j, k + 1, zb) - ex) * idz;
    float dEz_dx = (ld(Ez, g, i + 1, j, k, zb) - ez) * idx;
    float dEy_dx = (ld(Ey, g, i + 1, j, k, zb) - ey) * idx;
    float dEx_dy = (ld(Ex, g, i, j + 1, k, zb) - ex) * idy;
    if (pml.on) {
        const float bx = pml.bB[0][i], by = pml.bB[1][j], bz = pml.bB[2][k];
        dEz_dy = cpml(pml.psiB + 0 * N, ix, by, dEz_dy);
        dEy_dz = cpml(pml.psiB + 1 * N, ix, bz, dEy_dz);
        dEx_dz = cpml(pml.psiB + 2 * N, ix, bz, dEx_dz);
        dEz_dx = cpml(pml.psiB + 3 * N, ix, bx, dEz_dx);
        dEy_dx = cpml(pml.psiB + 4 * N, ix, bx, dEy_dx);
        dEx_dy = cpml(pml.psiB + 5 * N, ix, by, dEx_dy);
    }
    f.B[ix] -= dtt * (dEz_dy - dEy_dz);
    f.B[N + ix] -= dtt * (dEx_dz - dEz_dx);
    f.B[2 * N + ix] -= dtt * (dEy_dx - dEx_dy);
}

// E += dt (curl B - J).  E_x at (i+1/2, j, k), E_y at (i, j+1/2, k), E_z at (i, j, k+1/2):
// backward differences of B.
__global__ void k_fdtd_e(FieldsDev f, GridDev g, PmlDev pml)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int zb = zblock(k, g.nzr);
    const long long N = g.ncell;
    const long long ix = ((long long)k * g.n[1] + j) * g.n[0] + i;
    const float *Bx = f.B, *By = f.B + N, *Bz = f.B + 2 * N;
    const float bxv = Bx[ix], byv = By[ix], bzv = Bz[ix];
    const float idx = 1.f / g.d[0], idy = 1.f / g.d[1], idz = 1.f / g.d[2];
    float dBz_dy = (bzv - ld(Bz, g, i, j - 1, k, zb)) * idy;
    float dBy_dz = (byv - ld(By, g, i, j, k - 1, zb)) * idz;
    float dBx_dz = (bxv - ld(Bx, g, i, j, k - 1, zb)) * idz;
    float dBz_dx = (bzv - ld(Bz, g, i - 1, j, k, zb)) * idx;
    float dBy_dx = (byv - ld(By, g, i - 1, j, k, zb)) * idx;
    float dBx_dy = (bxv - ld(Bx, g, i, j - 1, k, zb)) * idy;
    if (pml.on) {
        const float bx = pml.bE[0][i], by = pml.bE[1][j], bz = pml.bE[2][k];
        dBz_dy = cpml(pml.psiE + 0 * N, ix, by, dBz_dy);
        dBy_dz = cpml(pml.psiE + 1 * N, ix, bz, dBy_dz);
        dBx_dz = cpml(pml.psiE + 2 * N, ix, bz, dBx_dz);
        dBz_dx = cpml(pml.psiE + 3 * N, ix, bx, dBz_dx);
        dBy_dx = cpml(pml.psiE + 4 * N, ix, bx, dBy_dx);
        dBx_dy = cpml(pml.psiE + 5 * N, ix, by, dBx_dy);
    }
    const float dt = g.dt;
    f.E[ix] += dt * (dBz_dy - dBy_dz - f.J[ix]);
    f.E[N + ix] += dt * (dBx_dz - dBz_dx - f.J[N + ix]);
    f.E[2 * N + ix] += dt * (dBy_dx - dBx_dy - f.J[2 * N + ix]);
}

// Moving window: every array moves down one z plane, the front plane becomes zero.  One
// thread owns one (i, j) column of one array, so the in-place shift has no race.
__global__ void k_shift_fields(float *const *arrays, int n_arrays, int nx, int ny, int nz)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (col >= nx * ny || a >= n_arrays) return;
    float *A = arrays[a];
    const long long plane = (long long)nx * ny;
    for (int k = 0; k < nz - 1; k++) A[k * plane + col] = A[(k + 1) * plane + col];
    A[(long long)(nz - 1) * plane + col] = 0.f;
}

__global__ void k_sumsq(const float *a, long long n, double *partial)
{
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = a[i];
        s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = s;
    }
}

}  // namespace

cudaError_t launch_fdtd_b(pic_ctx *c, float dtt)
{
    dim3 blk(32, 8, 1), grd((c->n[0] + 31) / 32, (c->n[1] + 7) / 8, c->n[2]);
    k_fdtd_b<<<grd, blk, 0, c->stream>>>(FieldsDev{c->E, c->B, c->J}, grid_dev(c), pml_dev(c), dtt);
    c->kernels++;
    return cudaGetLastError();
}

cudaError_t launch_fdtd_e(pic_ctx *c)
{
    dim3 blk(32, 8, 1), grd((c->n[0] + 31) / 32, (c->n[1] + 7) / 8, c->n[2]);
    k_fdtd_e<<<grd, blk, 0, c->stream>>>(FieldsDev{c->E, c->B, c->J}, grid_dev(c), pml_dev(c));
    c->kernels++;
    return cudaGetLastError();
}

cudaError_t launch_shift_fields(pic_ctx *c)
{
    const int cols = c->n[0] * c->n[1];
    k_shift_fields<<<dim3((cols + 255) / 256, c->shift_n), 256, 0, c->stream>>>(c->shift_tab, c->shift_n, c->n[0],
                                                                                c->n[1], c->n[2]);
    c->kernels++;
    return cudaGetLastError();
}

// (1/2) sum (E^2 + B^2) dV over the grid, or over the rows of one run of an ensemble (run >= 0).
cudaError_t launch_field_energy(pic_ctx *c, double *out_host, int run)
{
    const int blocks = 1024;
    double acc = 0.0;
    std::vector<double> part(blocks);
    const long long plane = (long long)c->n[0] * c->n[1];
    const long long off = run < 0 ? 0 : (long long)run * c->nzr * plane;
    const long long len = run < 0 ? c->ncell : (long long)c->nzr * plane;
    for (int q = 0; q < 6; q++) {
        const float *a = (q < 3 ? c->E + q * c->ncell : c->B + (q - 3) * c->ncell) + off;
        k_sumsq<<<blocks, 256, 0, c->stream>>>(a, len, c->red);
        c->kernels++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(part.data(), c->red, blocks * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return e;
        for (int b = 0; b < blocks; b++) acc += part[b];
    }
    *out_host = 0.5 * acc * c->d[0] * c->d[1] * c->d[2];
    return cudaSuccess;
}

}  // namespace gbpic
