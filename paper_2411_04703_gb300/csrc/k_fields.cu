// Yee FDTD update of Maxwell's equations in the RRF (Eq. Max1-Max2 normalised: dE/dt =
// curl B - J, dB/dt = -curl E), with B split into two half steps so that E^n and B^n are
// co-timed at the particle gather, and a convolutional PML (kappa = 1, alpha = 0) in the
// absorbing slabs ("the fields are absorbed upon interaction with the boundaries").
// One thread per (i, j) column of KZ cells, x fastest across a warp; neighbours outside a
// non-periodic face read as zero.
#include "gbpic_internal.cuh"

namespace gbpic {
namespace {

// CPML-stretched derivative dF + psi' with psi' = b psi + (b - 1) dF (psi the value loaded
// before; b >= 1: outside the layers, no auxiliary term).  The new psi' is returned in psi.
__device__ __forceinline__ float cpml_d(float b, float &psi, float dF)
{
    if (b >= 1.f) return dF;
    psi = fmaf(b, psi, (b - 1.f) * dF);
    return dF + psi;
}

// Cells per thread along z.  A thread walks KZ consecutive cells of one (i, j) column, so the
// z-neighbour it needs for one cell is a value it loads for the next (or loaded for the previous)
// one, and its x and y neighbour offsets (with the face rules) are worked out once per column.
// Six 256-thread blocks per SM (40 registers) keep more loads in flight than four at 64; both
// measured faster than one thread per cell, which spent ~375 instructions a cell on index and
// face arithmetic.
constexpr int kFdtdKzB = 8;
constexpr int kFdtdKzE = 8;

// Offset of the neighbour at p + s (s = +1 or -1) of a dim of n cells with stride st: within the
// grid the plain offset, across a periodic face the wrapped one (n = 1: the cell itself), across
// another face none (ok = false: the neighbour reads as zero).
__device__ __forceinline__ long long nb_off(int p, int s, int n, bool per, long long st, bool &ok)
{
    ok = true;
    const int q = p + s;
    if (q >= 0 && q < n) return s * st;
    if (!per) { ok = false; return 0; }
    return (long long)(pwrap(q, n) - p) * st;
}

__device__ __forceinline__ float ldo(const float *__restrict__ F, long long ix, long long off, bool ok)
{
    return ok ? __ldg(F + ix + off) : 0.f;
}

// B -= dtt curl E (half step).  B_x at (i, j+1/2, k+1/2), B_y at (i+1/2, j, k+1/2),
// B_z at (i+1/2, j+1/2, k): forward differences of E.  Every load of a cell (E and its
// neighbours, B, the layers' psi) is issued before its first store.
template <int KZ>
__global__ void __launch_bounds__(256, 6) k_fdtd_b(const float *__restrict__ E, float *__restrict__ B,
                                                float *__restrict__ psiB, GridDev g, PmlDev pml, float dtt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z * KZ;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const long long N = g.ncell, nx = g.n[0], nxy = (long long)g.n[0] * g.n[1];
    const float *Ex = E, *Ey = E + N, *Ez = E + 2 * N;
    bool okx, oky;
    const long long ox = nb_off(i, 1, g.n[0], g.periodic[0], 1, okx);
    const long long oy = nb_off(j, 1, g.n[1], g.periodic[1], nx, oky);
    const float idx = 1.f / g.d[0], idy = 1.f / g.d[1], idz = 1.f / g.d[2];
    const float bx = pml.on ? pml.bB[0][i] : 1.f, by = pml.on ? pml.bB[1][j] : 1.f;
    const int kend = min(k0 + KZ, g.n[2]);
    int zb = zblock(k0, g.nzr);
    long long ix = k0 * nxy + j * nx + i;
    float ex = Ex[ix], ey = Ey[ix];
    for (int k = k0; k < kend; k++, ix += nxy) {
        if (k >= zb + g.nzr) zb += g.nzr;
        bool okz;
        const long long oz = nb_off(k - zb, 1, g.nzr, g.periodic[2], nxy, okz);
        const float ez = Ez[ix];
        const float ez_y = ldo(Ez, ix, oy, oky), ey_z = ldo(Ey, ix, oz, okz);
        const float ex_z = ldo(Ex, ix, oz, okz), ez_x = ldo(Ez, ix, ox, okx);
        const float ey_x = ldo(Ey, ix, ox, okx), ex_y = ldo(Ex, ix, oy, oky);
        const float b0 = B[ix], b1 = B[N + ix], b2 = B[2 * N + ix];
        float dEz_dy = (ez_y - ez) * idy;
        float dEy_dz = (ey_z - ey) * idz;
        float dEx_dz = (ex_z - ex) * idz;
        float dEz_dx = (ez_x - ez) * idx;
        float dEy_dx = (ey_x - ey) * idx;
        float dEx_dy = (ex_y - ex) * idy;
        if (pml.on) {
            const float bz = pml.bB[2][k];
            if (bx < 1.f || by < 1.f || bz < 1.f) {
                float p[6];
#pragma unroll
                for (int q = 0; q < 6; q++) p[q] = psiB[q * N + ix];
                dEz_dy = cpml_d(by, p[0], dEz_dy);
                dEy_dz = cpml_d(bz, p[1], dEy_dz);
                dEx_dz = cpml_d(bz, p[2], dEx_dz);
                dEz_dx = cpml_d(bx, p[3], dEz_dx);
                dEy_dx = cpml_d(bx, p[4], dEy_dx);
                dEx_dy = cpml_d(by, p[5], dEx_dy);
                if (by < 1.f) { psiB[0 * N + ix] = p[0]; psiB[5 * N + ix] = p[5]; }
                if (bz < 1.f) { psiB[1 * N + ix] = p[1]; psiB[2 * N + ix] = p[2]; }
                if (bx < 1.f) { psiB[3 * N + ix] = p[3]; psiB[4 * N + ix] = p[4]; }
            }
        }
        B[ix] = b0 - dtt * (dEz_dy - dEy_dz);
        B[N + ix] = b1 - dtt * (dEx_dz - dEz_dx);
        B[2 * N + ix] = b2 - dtt * (dEy_dx - dEx_dy);
        // the next cell's own E_x, E_y are this cell's z neighbours, unless this cell's z
        // neighbour was a wrap or a zero (the last row of a run)
        if (okz && oz == nxy) { ex = ex_z; ey = ey_z; }
        else if (k + 1 < kend) { ex = Ex[ix + nxy]; ey = Ey[ix + nxy]; }
    }
}

// E += dt (curl B - J).  E_x at (i+1/2, j, k), E_y at (i, j+1/2, k), E_z at (i, j, k+1/2):
// backward differences of B.  Loads first, as in k_fdtd_b.
template <int KZ>
__global__ void __launch_bounds__(256, 6) k_fdtd_e(float *__restrict__ E, const float *__restrict__ B,
                                                const float *__restrict__ J, float *__restrict__ psiE, GridDev g,
                                                PmlDev pml)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z * KZ;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const long long N = g.ncell, nx = g.n[0], nxy = (long long)g.n[0] * g.n[1];
    const float *Bx = B, *By = B + N, *Bz = B + 2 * N;
    bool okx, oky;
    const long long ox = nb_off(i, -1, g.n[0], g.periodic[0], 1, okx);
    const long long oy = nb_off(j, -1, g.n[1], g.periodic[1], nx, oky);
    const float idx = 1.f / g.d[0], idy = 1.f / g.d[1], idz = 1.f / g.d[2];
    const float bx = pml.on ? pml.bE[0][i] : 1.f, by = pml.on ? pml.bE[1][j] : 1.f;
    const float dt = g.dt;
    const int kend = min(k0 + KZ, g.n[2]);
    int zb = zblock(k0, g.nzr);
    long long ix = k0 * nxy + j * nx + i;
    float bx_z = 0.f, by_z = 0.f;   // B_x, B_y of the cell below (loaded with the cell itself)
    bool below = false;              // they hold the row k - 1 of the walk
    for (int k = k0; k < kend; k++, ix += nxy) {
        if (k >= zb + g.nzr) { zb += g.nzr; below = false; }
        const float bxv = Bx[ix], byv = By[ix], bzv = Bz[ix];
        if (!below) {
            bool okz;
            const long long oz = nb_off(k - zb, -1, g.nzr, g.periodic[2], nxy, okz);
            bx_z = ldo(Bx, ix, oz, okz);
            by_z = ldo(By, ix, oz, okz);
        }
        const float bz_y = ldo(Bz, ix, oy, oky), bz_x = ldo(Bz, ix, ox, okx);
        const float by_x = ldo(By, ix, ox, okx), bx_y = ldo(Bx, ix, oy, oky);
        const float e0 = E[ix], e1 = E[N + ix], e2 = E[2 * N + ix];
        const float j0 = J[ix], j1 = J[N + ix], j2 = J[2 * N + ix];
        float dBz_dy = (bzv - bz_y) * idy;
        float dBy_dz = (byv - by_z) * idz;
        float dBx_dz = (bxv - bx_z) * idz;
        float dBz_dx = (bzv - bz_x) * idx;
        float dBy_dx = (byv - by_x) * idx;
        float dBx_dy = (bxv - bx_y) * idy;
        if (pml.on) {
            const float bz = pml.bE[2][k];
            if (bx < 1.f || by < 1.f || bz < 1.f) {
                float p[6];
#pragma unroll
                for (int q = 0; q < 6; q++) p[q] = psiE[q * N + ix];
                dBz_dy = cpml_d(by, p[0], dBz_dy);
                dBy_dz = cpml_d(bz, p[1], dBy_dz);
                dBx_dz = cpml_d(bz, p[2], dBx_dz);
                dBz_dx = cpml_d(bx, p[3], dBz_dx);
                dBy_dx = cpml_d(bx, p[4], dBy_dx);
                dBx_dy = cpml_d(by, p[5], dBx_dy);
                if (by < 1.f) { psiE[0 * N + ix] = p[0]; psiE[5 * N + ix] = p[5]; }
                if (bz < 1.f) { psiE[1 * N + ix] = p[1]; psiE[2 * N + ix] = p[2]; }
                if (bx < 1.f) { psiE[3 * N + ix] = p[3]; psiE[4 * N + ix] = p[4]; }
            }
        }
        E[ix] = e0 + dt * (dBz_dy - dBy_dz - j0);
        E[N + ix] = e1 + dt * (dBx_dz - dBz_dx - j1);
        E[2 * N + ix] = e2 + dt * (dBy_dx - dBx_dy - j2);
        // this cell's B_x, B_y are the next cell's z neighbours below (B is not written here)
        bx_z = bxv;
        by_z = byv;
        below = true;
    }
}

// Artificial neutralising ions: the z prefix G(i, j, k) = -dz sum_{k' <= k} rho'(i, j, k') of the
// compensated species' density (relative to the column mean on a periodic z), FP64 along each
// column.  The ions' current while they fade over T is J_z = G / T (div J = -d rho_ion / dt).
__global__ void k_ion_prefix(const float *rho, float *G, int nx, int ny, int nz, double dz, int zper)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= nx * ny) return;
    const long long plane = (long long)nx * ny;
    double mean = 0.0;
    if (zper) {
        for (int k = 0; k < nz; k++) mean += rho[k * plane + col];
        mean /= (double)nz;
    }
    double acc = 0.0;
    for (int k = 0; k < nz; k++) {
        acc += (double)rho[k * plane + col] - mean;
        G[k * plane + col] = (float)(-dz * acc);
    }
}

__global__ void k_ion_current(float *Jz, const float *G, long long n, float f)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Jz[i] += f * G[i];
}

// Moving window with artificial ions: the prefix of the shifted density is the old prefix one
// plane up minus the dropped plane's part; no ions enter at the front.
__global__ void k_ion_shift(float *G, int nx, int ny, int nz)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= nx * ny) return;
    const long long plane = (long long)nx * ny;
    const float g0 = G[col];
    for (int k = 0; k + 1 < nz; k++) G[k * plane + col] = G[(k + 1) * plane + col] - g0;
    if (nz > 1) G[(long long)(nz - 1) * plane + col] = G[(long long)(nz - 2) * plane + col];
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
    dim3 blk(32, 8, 1), grd((c->n[0] + 31) / 32, (c->n[1] + 7) / 8, (c->n[2] + kFdtdKzB - 1) / kFdtdKzB);
    const PmlDev pml = pml_dev(c);
    k_fdtd_b<kFdtdKzB><<<grd, blk, 0, c->stream>>>(c->E, c->B, pml.psiB, grid_dev(c), pml, dtt);
    c->kernels++;
    return cudaGetLastError();
}

cudaError_t launch_fdtd_e(pic_ctx *c)
{
    dim3 blk(32, 8, 1), grd((c->n[0] + 31) / 32, (c->n[1] + 7) / 8, (c->n[2] + kFdtdKzE - 1) / kFdtdKzE);
    const PmlDev pml = pml_dev(c);
    k_fdtd_e<kFdtdKzE><<<grd, blk, 0, c->stream>>>(c->E, c->B, c->J, pml.psiE, grid_dev(c), pml);
    c->kernels++;
    return cudaGetLastError();
}

cudaError_t launch_ion_prefix(pic_ctx *c, const float *rho, float *G)
{
    const int cols = c->n[0] * c->n[1];
    k_ion_prefix<<<(cols + 255) / 256, 256, 0, c->stream>>>(rho, G, c->n[0], c->n[1], c->n[2], c->d[2],
                                                           c->bc[2][0] == PIC_BC_PERIODIC);
    c->kernels++;
    return cudaGetLastError();
}

cudaError_t launch_ion_current(pic_ctx *c, float f)
{
    k_ion_current<<<c->num_sms * 4, 256, 0, c->stream>>>(c->J + 2 * c->ncell, c->ion_G, c->ncell, f);
    c->kernels++;
    return cudaGetLastError();
}

cudaError_t launch_ion_shift(pic_ctx *c)
{
    const int cols = c->n[0] * c->n[1];
    k_ion_shift<<<(cols + 255) / 256, 256, 0, c->stream>>>(c->ion_G, c->n[0], c->n[1], c->n[2]);
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
