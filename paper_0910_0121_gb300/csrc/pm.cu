// PM (long-range) part of the TreePM split (Sec. 2.1-2.2 step 1; Table 2 rows "density
// assignment", "FFT", "convolution", "force interpolation").
//
// The PP part is Newton's law times g_P3M (Eq. 1-2), i.e. Newton's law minus the force
// between two S2 clouds of radius eta; the PM part carries exactly that cloud-cloud force:
//   phi_k = G(k) rho_k,  G(k) = -4 pi S(k eta)^2 / (k^2 W(k)^2),  k = 0 removed,
// with S(xi) = 12 (2 - 2 cos xi - xi sin xi)/xi^4 and W the assignment window (CIC p = 2,
// TSC p = 3, divided out once for the assignment and once for the interpolation).  The
// acceleration is -i k phi_k per component (Nyquist components zeroed), transformed back
// and interpolated with the assignment weights.  Grid points sit at x = j L/n (periodic).
//
// G is tabulated once per (n, L, r_cut, scheme) in FP64 over |k_x|, |k_y|, k_z (the
// (n/2+1)^3 table the paper also keeps, Sec. 3.2.5), with 1/Delta^3 (mass -> density)
// and 1/n^3 (unnormalised inverse FFT) folded in.  The FFTs are cuFFT (FP32).
#include <cufft.h>

#include "common.cuh"
#include "pm.cuh"

namespace greem {

struct PmGeom {
    int n;             // grid points per side
    int scheme;        // 0 CIC, 1 TSC
    double L;
    double inv_delta;  // n / L
    int pow2_e;        // L = 2^pow2_e, or kNotPow2
    int log2n;         // n = 2^log2n, or -1
};

// Integer grid index and fractional part of x * n / L (x wrapped into [0, L)).
__device__ __forceinline__ void grid_coord(double x, const PmGeom &g, int &i, float &f)
{
    x = wrap_pos_fast(x, g.L);
    if (g.pow2_e != kNotPow2 && g.log2n >= 0) {
        // exact: x n/L = fixed52(x) * 2^(log2n - 52)
        const long long q = fixed52(x, g.pow2_e);
        const int sh = 52 - g.log2n;
        i = (int)(q >> sh);
        f = __ll2float_rn(q & ((1ll << sh) - 1)) * __int_as_float((127 - sh) << 23);
    } else {
        const double s = x * g.inv_delta;
        const double fl = floor(s);
        i = (int)fl;
        f = (float)(s - fl);
    }
    if (i >= g.n) {  // x * n / L rounded up to n
        i -= g.n;
    }
}

// Per-axis weights: CIC (i, i+1) with (1-f, f); TSC (i-1, i, i+1) about the nearest point.
template <int SCHEME>
__device__ __forceinline__ void axis_weights(int i, float f, int n, int (&idx)[3], float (&w)[3])
{
    if (SCHEME == 0) {
        idx[0] = i;
        idx[1] = i + 1 == n ? 0 : i + 1;
        w[0] = 1.0f - f;
        w[1] = f;
        idx[2] = 0;
        w[2] = 0.0f;
    } else {
        int c = i;
        float d = f;
        if (f >= 0.5f) {
            c = i + 1 == n ? 0 : i + 1;
            d = f - 1.0f;
        }
        idx[0] = c == 0 ? n - 1 : c - 1;
        idx[1] = c;
        idx[2] = c + 1 == n ? 0 : c + 1;
        const float a = 0.5f - d, b = 0.5f + d;
        w[0] = 0.5f * a * a;
        w[1] = 0.75f - d * d;
        w[2] = 0.5f * b * b;
    }
}

// Position of particle p: from AoS input (pos != null) or from sorted SoA.
__device__ __forceinline__ void particle_pos(const double *pos, const double *xs, const double *ys, const double *zs,
                                             uint32_t p, double &x, double &y, double &z)
{
    if (pos) {
        x = pos[3 * (size_t)p];
        y = pos[3 * (size_t)p + 1];
        z = pos[3 * (size_t)p + 2];
    } else {
        x = xs[p];
        y = ys[p];
        z = zs[p];
    }
}

template <int SCHEME>
__global__ void __launch_bounds__(256) k_pm_assign(const double *__restrict__ pos, const double *__restrict__ xs,
                                                   const double *__restrict__ ys, const double *__restrict__ zs,
                                                   const float *__restrict__ mass, uint32_t N, PmGeom g,
                                                   float *__restrict__ grid)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    double x, y, z;
    particle_pos(pos, xs, ys, zs, p, x, y, z);
    int ix, iy, iz;
    float fx, fy, fz;
    grid_coord(x, g, ix, fx);
    grid_coord(y, g, iy, fy);
    grid_coord(z, g, iz, fz);
    int jx[3], jy[3], jz[3];
    float wx[3], wy[3], wz[3];
    axis_weights<SCHEME>(ix, fx, g.n, jx, wx);
    axis_weights<SCHEME>(iy, fy, g.n, jy, wy);
    axis_weights<SCHEME>(iz, fz, g.n, jz, wz);
    const float m = mass[p];
    constexpr int K = SCHEME == 0 ? 2 : 3;
    const size_t n = (size_t)g.n;
#pragma unroll
    for (int a = 0; a < K; a++)
#pragma unroll
        for (int b = 0; b < K; b++) {
            const float mab = m * wx[a] * wy[b];
            float *row = grid + ((size_t)jx[a] * n + (size_t)jy[b]) * n;
#pragma unroll
            for (int c = 0; c < K; c++) atomicAdd(row + jz[c], mab * wz[c]);
        }
}

template <int SCHEME>
__global__ void __launch_bounds__(256) k_pm_interp(const double *__restrict__ pos, const double *__restrict__ xs,
                                                   const double *__restrict__ ys, const double *__restrict__ zs,
                                                   const uint32_t *__restrict__ perm, uint32_t N, PmGeom g,
                                                   const float *__restrict__ grid, int comp, int accumulate,
                                                   float *__restrict__ acc)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    double x, y, z;
    particle_pos(pos, xs, ys, zs, p, x, y, z);
    int ix, iy, iz;
    float fx, fy, fz;
    grid_coord(x, g, ix, fx);
    grid_coord(y, g, iy, fy);
    grid_coord(z, g, iz, fz);
    int jx[3], jy[3], jz[3];
    float wx[3], wy[3], wz[3];
    axis_weights<SCHEME>(ix, fx, g.n, jx, wx);
    axis_weights<SCHEME>(iy, fy, g.n, jy, wy);
    axis_weights<SCHEME>(iz, fz, g.n, jz, wz);
    constexpr int K = SCHEME == 0 ? 2 : 3;
    const size_t n = (size_t)g.n;
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < K; a++)
#pragma unroll
        for (int b = 0; b < K; b++) {
            const float *row = grid + ((size_t)jx[a] * n + (size_t)jy[b]) * n;
            float t = 0.0f;
#pragma unroll
            for (int c = 0; c < K; c++) t = fmaf(wz[c], __ldg(row + jz[c]), t);
            s = fmaf(wx[a] * wy[b], t, s);
        }
    const size_t o = (size_t)(perm ? perm[p] : p) * 3 + comp;
    acc[o] = accumulate ? acc[o] + s : s;
}

// Green's table over (|m_x|, |m_y|, m_z) in [0, n/2]^3, FP64 then rounded to FP32.
__global__ void k_pm_table(int n, double L, double eta, int scheme, float *__restrict__ table)
{
    const int h = n / 2 + 1;
    const long long total = (long long)h * h * h;
    const double pi = 3.14159265358979323846;
    const double delta = L / n;
    const double norm = 1.0 / (delta * delta * delta) / ((double)n * n * n);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / ((long long)h * h)), b = (int)((t / h) % h), c = (int)(t % h);
        if (a == 0 && b == 0 && c == 0) {
            table[t] = 0.0f;
            continue;
        }
        const double kx = 2 * pi * a / L, ky = 2 * pi * b / L, kz = 2 * pi * c / L;
        const double k2 = kx * kx + ky * ky + kz * kz;
        const double xi = sqrt(k2) * eta;
        double S;
        if (xi < 1e-2) {
            S = 1.0 - xi * xi / 15.0 + xi * xi * xi * xi / 560.0;
        } else {
            S = 12.0 * (2.0 - 2.0 * cos(xi) - xi * sin(xi)) / (xi * xi * xi * xi);
        }
        auto sinc = [](double v) { return v == 0.0 ? 1.0 : sin(v) / v; };
        double W = sinc(0.5 * kx * delta) * sinc(0.5 * ky * delta) * sinc(0.5 * kz * delta);
        W = scheme == 0 ? W * W : W * W * W;
        table[t] = (float)(-4.0 * pi * S * S / (k2 * W * W) * norm);
    }
}

// phi_k = rho_k * G, in place on the half-complex spectrum [n][n][n/2+1].
__global__ void __launch_bounds__(256) k_pm_convolve(cufftComplex *__restrict__ spec, int n,
                                                     const float *__restrict__ table)
{
    const int hz = n / 2 + 1, h = n / 2 + 1;
    const long long total = (long long)n * n * hz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t / ((long long)n * hz)), y = (int)((t / hz) % n), z = (int)(t % hz);
        const int ax = x <= n / 2 ? x : n - x, ay = y <= n / 2 ? y : n - y;
        const float gk = table[((long long)ax * h + ay) * h + z];
        cufftComplex v = spec[t];
        v.x *= gk;
        v.y *= gk;
        spec[t] = v;
    }
}

// out = -i k_comp phi_k (the Nyquist component of k_comp is zero).
__global__ void __launch_bounds__(256) k_pm_gradient(const cufftComplex *__restrict__ phi, int n, double L, int comp,
                                                     cufftComplex *__restrict__ out)
{
    const int hz = n / 2 + 1;
    const long long total = (long long)n * n * hz;
    const float twopi_L = (float)(2.0 * 3.14159265358979323846 / L);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t / ((long long)n * hz)), y = (int)((t / hz) % n), z = (int)(t % hz);
        int m = comp == 0 ? x : (comp == 1 ? y : z);
        if (comp < 2) m = m < n / 2 ? m : (m == n / 2 ? 0 : m - n);
        else m = m == n / 2 ? 0 : m;
        const float k = twopi_L * (float)m;
        const cufftComplex v = phi[t];
        cufftComplex r;
        r.x = k * v.y;
        r.y = -k * v.x;
        out[t] = r;
    }
}

int pm_plan(PmPlan &pl, int n, cudaStream_t s)
{
    if (pl.have && pl.n == n) {
        cufftSetStream(pl.r2c, s);
        cufftSetStream(pl.c2r, s);
        return 0;
    }
    if (pl.have) {
        cufftDestroy(pl.r2c);
        cufftDestroy(pl.c2r);
        pl.have = false;
    }
    if (cufftPlan3d(&pl.r2c, n, n, n, CUFFT_R2C) != CUFFT_SUCCESS) return -1;
    if (cufftPlan3d(&pl.c2r, n, n, n, CUFFT_C2R) != CUFFT_SUCCESS) {
        cufftDestroy(pl.r2c);
        return -1;
    }
    cufftSetStream(pl.r2c, s);
    cufftSetStream(pl.c2r, s);
    pl.n = n;
    pl.have = true;
    return 0;
}

void pm_plan_destroy(PmPlan &pl)
{
    if (pl.have) {
        cufftDestroy(pl.r2c);
        cufftDestroy(pl.c2r);
    }
    pl.have = false;
}

void launch_pm_table(int n, double L, double r_cut, int scheme, float *table, cudaStream_t s, int nsm)
{
    k_pm_table<<<nsm * 8, 256, 0, s>>>(n, L, 0.5 * r_cut, scheme, table);
    g_launches++;
}

// The whole PM force: grid n^3 floats, spec and tmp n*n*(n/2+1) complex, table from
// launch_pm_table.  Positions from AoS pos (input order, perm null) or sorted SoA
// xs/ys/zs with perm (sorted -> input index).  acc gets (or accumulates) input order.
int run_pm(const PmPlan &pl, const double *pos, const double *xs, const double *ys, const double *zs,
           const float *mass, const uint32_t *perm, uint32_t N, double L, int n, int scheme, int pow2_e,
           const float *table, float *grid, cufftComplex *spec, cufftComplex *tmp, float *acc, int accumulate,
           cudaStream_t s, int nsm)
{
    PmGeom g;
    g.n = n;
    g.scheme = scheme;
    g.L = L;
    g.inv_delta = n / L;
    g.pow2_e = pow2_e;
    int lg = -1;
    for (int q = 0; q < 31; q++)
        if ((1 << q) == n) lg = q;
    g.log2n = lg;
    const size_t cells = (size_t)n * n * n;
    cudaMemsetAsync(grid, 0, cells * sizeof(float), s);
    const unsigned pb = (N + 255) / 256;
    if (scheme == 0) k_pm_assign<0><<<pb, 256, 0, s>>>(pos, xs, ys, zs, mass, N, g, grid);
    else k_pm_assign<1><<<pb, 256, 0, s>>>(pos, xs, ys, zs, mass, N, g, grid);
    g_launches++;
    if (cufftExecR2C(pl.r2c, grid, spec) != CUFFT_SUCCESS) return -2;
    k_pm_convolve<<<nsm * 8, 256, 0, s>>>(spec, n, table);
    g_launches++;
    for (int comp = 0; comp < 3; comp++) {
        k_pm_gradient<<<nsm * 8, 256, 0, s>>>(spec, n, L, comp, tmp);
        g_launches++;
        if (cufftExecC2R(pl.c2r, tmp, grid) != CUFFT_SUCCESS) return -2;
        if (scheme == 0) k_pm_interp<0><<<pb, 256, 0, s>>>(pos, xs, ys, zs, perm, N, g, grid, comp, accumulate, acc);
        else k_pm_interp<1><<<pb, 256, 0, s>>>(pos, xs, ys, zs, perm, N, g, grid, comp, accumulate, acc);
        g_launches++;
    }
    return 0;
}

}  // namespace greem
