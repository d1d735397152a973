// Time integration (Sec. 2.2 steps 1, 6 and 7; Sec. 2.4): kick, drift, the shared
// adaptive timestep of Eq. 7, the shared softening of Eq. 6, and the comoving kick and
// drift factors.
//
// Each kernel is a plain sequence of correctly rounded operations (no fused multiply-add),
// so that the same operations in numpy give identical bits.
#include "common.cuh"

#include <cmath>

namespace greem {

// v += f a (FP32, component by component).
__global__ void __launch_bounds__(256) k_kick(float *__restrict__ vel, const float *__restrict__ acc, size_t n3,
                                              float f)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x)
        vel[i] = __fadd_rn(vel[i], __fmul_rn(f, acc[i]));
}

// x += f v in FP64, wrapped into [0, L) by the same rule as the keys.
__global__ void __launch_bounds__(256) k_drift(double *__restrict__ pos, const float *__restrict__ vel, size_t n3,
                                               double f, double L)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x)
        pos[i] = wrap_pos_fast(__dadd_rn(pos[i], __dmul_rn(f, (double)vel[i])), L);
}

// Largest |v|^2 and |a|^2 over the particles, (x^2 + y^2) + z^2 in FP32; non-negative
// floats order like their bit patterns, so an integer max finds them.
__global__ void __launch_bounds__(256) k_vmax_amax(const float *__restrict__ vel, const float *__restrict__ acc,
                                                   uint32_t N, unsigned int *__restrict__ out)
{
    float vm = 0.f, am = 0.f;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float *v = vel + 3 * (size_t)i, *a = acc + 3 * (size_t)i;
        const float v2 = __fadd_rn(__fadd_rn(__fmul_rn(v[0], v[0]), __fmul_rn(v[1], v[1])), __fmul_rn(v[2], v[2]));
        const float a2 = __fadd_rn(__fadd_rn(__fmul_rn(a[0], a[0]), __fmul_rn(a[1], a[1])), __fmul_rn(a[2], a[2]));
        vm = fmaxf(vm, v2);
        am = fmaxf(am, a2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, __float_as_uint(vm));
        atomicMax(out + 1, __float_as_uint(am));
    }
}

void launch_kick(float *vel, const float *acc, uint32_t N, float f, cudaStream_t s, int nsm)
{
    k_kick<<<nsm * 8, 256, 0, s>>>(vel, acc, 3 * (size_t)N, f);
    g_launches++;
}

void launch_drift(double *pos, const float *vel, uint32_t N, double f, double L, cudaStream_t s, int nsm)
{
    k_drift<<<nsm * 8, 256, 0, s>>>(pos, vel, 3 * (size_t)N, f, L);
    g_launches++;
}

void launch_vmax_amax(const float *vel, const float *acc, uint32_t N, unsigned int *out, cudaStream_t s, int nsm)
{
    cudaMemsetAsync(out, 0, 2 * sizeof(unsigned int), s);
    k_vmax_amax<<<nsm * 4, 256, 0, s>>>(vel, acc, N, out);
    g_launches++;
}

// ---------------------------------------------------------------- host helpers
// Eq. 7: zeta * min(sqrt(eps / max|a|), eps / max|v|) from the squared maxima; a term
// whose maximum is 0 sets no bound (+inf when both are 0).
double timestep_eq7(double eps, double zeta, float v2max, float a2max)
{
    double dt = INFINITY;
    if (a2max > 0.f) dt = std::fmin(dt, std::sqrt(eps / std::sqrt((double)a2max)));
    if (v2max > 0.f) dt = std::fmin(dt, eps / std::sqrt((double)v2max));
    return zeta * dt;
}

// Eq. 6 read as the physical softening: (1+z_crit)/(1+z) eps_fin above z_crit (constant
// in comoving coordinates, eps_fin (1+z_crit)), eps_fin below (constant physically).
double softening_eq6(double eps_fin, double z_crit, double z)
{
    return z >= z_crit ? (1.0 + z_crit) / (1.0 + z) * eps_fin : eps_fin;
}

// int_{a0}^{a1} da / (a^p H(a)), H = H0 sqrt(om a^-3 + (1 - om - ol) a^-2 + ol), by
// composite Gauss-Legendre (4 nodes) on 4096 intervals: kick p = 2 (int dt/a), drift
// p = 3 (int dt/a^2).
double cosmo_integral(double a0, double a1, double om, double ol, double h0, int p)
{
    static const double xg[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563, 0.8611363115940526};
    static const double wg[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461, 0.3478548451374538};
    const int n = 4096;
    const double h = (a1 - a0) / n, ok = 1.0 - om - ol;
    double sum = 0.0;
    for (int i = 0; i < n; i++) {
        const double c = a0 + (i + 0.5) * h;
        for (int q = 0; q < 4; q++) {
            const double a = c + 0.5 * h * xg[q];
            const double H = h0 * std::sqrt(om / (a * a * a) + ok / (a * a) + ol);
            sum += wg[q] * 0.5 * h / (std::pow(a, p) * H);
        }
    }
    return sum;
}

}  // namespace greem
