// S6 pairwise cutoff force over the interaction lists (Sec. 2.1 Eq. 1-2; Sec. 3.1.1).
//
// FP32 kernel.  Positions are in units of r_cut = 2 eta relative to the group's cell
// centre (the list builder did the FP64 work), so with xi = r/r_cut and R = r/eta = 2 xi
//   acc_i = (1/r_cut^2) sum_j m_j g(2 xi) D / xi^3 ,   D = X_j - X_i .
// Eq. 2 is evaluated without cancellation.  Its outer branch factors exactly as
//   g(R) = (2-R)^5 (7R^3 + 22R^2 + 10R + 4) / 140            (1 <= R < 2),
// and the inner branch is the outer one plus (1-R)^6 (7R^2 + 18R + 3) / 35, so with
// v = saturate(1 - R/2) = saturate(1 - xi) and u = saturate(1 - R) = saturate(2v - 1)
//   g(R) = v^5 C(R) + u^6 P(R),  C = (8/35)(7R^3 + 22R^2 + 10R + 4),  P = (7R^2 + 18R + 3)/35,
// a sum of two non-negative terms for every R >= 0 that is exactly 0 for R >= 2.  The
// relative error of g therefore stays at a few ulp even where g -> 0 near the cutoff.
// The kernels need g(2 xi)/xi^3 = v^5 C(2 xi)/xi^3 + u^6 P(2 xi)/xi^3, and with w = 1/xi
// both quotients are polynomials in w with positive coefficients:
//   Chat(w) = (8/35)(4w^3 + 20w^2 + 88w + 56),   Phat(w) = (3w^3 + 36w^2 + 28w)/35,
// evaluated by Horner's rule.  v comes from r^2 and w without forming xi.
//
// Two forms of the pair loop.  With an even number I of i-particles per lane, pairs of
// i-particles share the sm_100-family packed FP32x2 instructions (two FP32 operations
// per instruction: half the issue slots, the FP32 pipe is then the limit); r^2 gets a
// floor of 2^-60 r_cut^2, so a pair at distance 0 (the particle itself, a coincident one)
// adds exactly 0 without a select.  With odd I the scalar loop runs and such a pair is
// selected out.
//
// Layout.  A persistent grid; each warp takes one group at a time from an atomic
// queue.  The warp's 32 lanes are split into S parts (S in 1, 2, ..., 32) of 32/S lanes;
// each lane holds I i-particles in registers and each part runs over every S-th list
// entry, so small groups do not idle lanes; the parts are summed by shuffles at the end.
// The layout of each pass comes from a table built at compile time from a cost model.
// The group's list streams through a per-warp double buffer in shared memory filled by
// 1-D bulk asynchronous copies (cp.async.bulk, the TMA engine) that complete on an
// mbarrier; every entry is read by the part's lanes as one broadcast 16-byte load.
#include <atomic>

#include "common.cuh"

namespace greem {

// ------------------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase; false after `polls` polls (the caller records a timeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t polls)
{
    for (uint32_t it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Largest number of i-particles a lane holds in one pass, and the launch bounds of the
// force kernel (registers per thread follow from them).
#ifndef GREEM_FORCE_IMAX
#define GREEM_FORCE_IMAX 6
#endif
#ifndef GREEM_FORCE_THREADS
#define GREEM_FORCE_THREADS 512
#endif
#ifndef GREEM_FORCE_MINB
#define GREEM_FORCE_MINB 1
#endif
#ifndef GREEM_FORCE_UNROLL
#define GREEM_FORCE_UNROLL 4
#endif
constexpr int kImax = GREEM_FORCE_IMAX;
constexpr int kUnroll = GREEM_FORCE_UNROLL;

// ------------------------------------------------------------------ Eq. 2 constants
// Chat(w) = ((kA3 w + kA2) w + kA1) w + kA0 and Phat(w) = ((kB3 w + kB2) w + kB1) w; the
// same numbers in reverse order give C(2 xi) = ((kA0 xi + kA1) xi + kA2) xi + kA3 and
// P(2 xi) = (kB1 xi + kB2) xi + kB3.
constexpr float kA0 = 12.8f;                    // 448/35
constexpr float kA1 = 20.11428571428571429f;    // 704/35
constexpr float kA2 = 4.571428571428571429f;    // 160/35
constexpr float kA3 = 0.9142857142857142857f;   //  32/35
constexpr float kB1 = 0.8f;                     //  28/35
constexpr float kB2 = 1.028571428571428571f;    //  36/35
constexpr float kB3 = 0.08571428571428571429f;  //   3/35

// saturate(a*b + c) and saturate(a + b) as single instructions (the .sat modifier clamps
// to [0, 1] and turns NaN into 0)
__device__ __forceinline__ float fma_sat(float a, float b, float c)
{
    float d;
    asm("fma.rn.ftz.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float add_sat(float a, float b)
{
    float d;
    asm("add.rn.ftz.sat.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// ------------------------------------------------------------------ packed FP32 pairs
// sm_100-family FP32x2 instructions: one instruction does the same operation on two FP32
// values held in a 64-bit register pair.  The FP32 pipe still takes two cycles for it,
// so the peak is unchanged, but the interaction needs half the issue slots and the FP32
// pipe, not instruction issue, becomes the limit.  Two i-particles share each packed
// value; the list entry is broadcast into both halves.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 rsqrt2(f32x2 v)
{
    float lo, hi;
    upk(v, lo, hi);
    asm("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(lo));
    asm("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(hi));
    return pk(lo, hi);
}
// r^2 gets 2^-60 (in r_cut^2) before the square root.  That is far below what FP32
// coordinates relative to the group centre resolve (~1e-7 r_cut), and it keeps w^3
// below 2^90, so a pair with D = 0 (the particle itself, a coincident particle) adds
// exactly 0 without a select; masses must stay below 2^38 for that (checked on input).
constexpr float kR2Floor = 8.673617379884035e-19f;  // 2^-60

// v = saturate(1 - xi) from r^2 and w = 1/xi, and u = saturate(2v - 1), as scalar
// saturating operations: the clamp rides on the FP32 instruction, where a packed
// operation and a separate max would take twice the issue slots (the packed forms
// have no .sat)
__device__ __forceinline__ void vu_pair(f32x2 r2, f32x2 w, f32x2 &v, f32x2 &u)
{
    float rl, rh, wl, wh;
    upk(r2, rl, rh);
    upk(w, wl, wh);
    const float vl = fma_sat(rl, -wl, 1.0f), vh = fma_sat(rh, -wh, 1.0f);
    v = pk(vl, vh);
    u = pk(fma_sat(vl, 2.0f, -1.0f), fma_sat(vh, 2.0f, -1.0f));
}

// Packed form of interact() for I = 2H i-particles: (xi[2h], xi[2h+1]) in xi2[h].
// 26 FP32 operations per pair (without softening) and one rsqrt.
template <int H, bool SOFT>
__device__ __forceinline__ void interact2(const float4 j, const f32x2 (&xi)[H], const f32x2 (&yi)[H],
                                          const f32x2 (&zi)[H], f32x2 (&ax)[H], f32x2 (&ay)[H], f32x2 (&az)[H],
                                          const f32x2 eps2)
{
    const f32x2 jx = pk(j.x, j.x), jy = pk(j.y, j.y), jz = pk(j.z, j.z), jm = pk(j.w, j.w);
    const f32x2 k[9] = {pk(kR2Floor, kR2Floor), pk(1.0f, 1.0f), pk(kA0, kA0), pk(kA1, kA1), pk(kA2, kA2),
                        pk(kA3, kA3),           pk(kB1, kB1),   pk(kB2, kB2), pk(kB3, kB3)};
#pragma unroll
    for (int h = 0; h < H; h++) {
        const f32x2 dx = sub2(jx, xi[h]), dy = sub2(jy, yi[h]), dz = sub2(jz, zi[h]);
        const f32x2 r2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, k[0])));
        const f32x2 w = rsqrt2(r2);
        f32x2 v, u;
        vu_pair(r2, w, v, u);
        const f32x2 v2 = mul2(v, v), v5 = mul2(mul2(v2, v2), v);
        const f32x2 u2 = mul2(u, u), u6 = mul2(mul2(u2, u2), u2);
        f32x2 sc;
        if (!SOFT) {
            // g(2 xi)/xi^3 = v^5 Chat(w) + u^6 Phat(w)
            const f32x2 cq = fma2(fma2(fma2(w, k[5], k[4]), w, k[3]), w, k[2]);
            const f32x2 pq = mul2(fma2(fma2(w, k[8], k[7]), w, k[6]), w);
            sc = mul2(jm, fma2(u6, pq, mul2(v5, cq)));
        } else {
            // Plummer softening: g at the unsoftened R = 2 xi times 1/(xi^2+eps^2)^(3/2)
            const f32x2 x = mul2(r2, w);
            const f32x2 c = fma2(fma2(fma2(x, k[2], k[3]), x, k[4]), x, k[5]);
            const f32x2 p = fma2(fma2(x, k[6], k[7]), x, k[8]);
            const f32x2 g = fma2(u6, p, mul2(v5, c));
            const f32x2 rs = rsqrt2(fma2(k[1], eps2, r2));
            sc = mul2(mul2(jm, g), mul2(mul2(rs, rs), rs));
        }
        ax[h] = fma2(sc, dx, ax[h]);
        ay[h] = fma2(sc, dy, ay[h]);
        az[h] = fma2(sc, dz, az[h]);
    }
}

template <int I, bool SOFT>
__device__ __forceinline__ void interact(const float4 j, const float (&xi)[I], const float (&yi)[I],
                                         const float (&zi)[I], float (&ax)[I], float (&ay)[I], float (&az)[I],
                                         float eps2)
{
#pragma unroll
    for (int s = 0; s < I; s++) {
        const float dx = j.x - xi[s], dy = j.y - yi[s], dz = j.z - zi[s];
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        // the same form as the packed loop; r^2 = 0 is selected out
        const float w = rsqrtf(r2);
        const float v = fma_sat(r2, -w, 1.0f), u = fma_sat(v, 2.0f, -1.0f);
        const float v2 = v * v, u2 = u * u;
        const float v5 = v2 * v2 * v, u6 = u2 * u2 * u2;
        float sc;
        if (!SOFT) {
            const float cq = fmaf(fmaf(fmaf(w, kA3, kA2), w, kA1), w, kA0);
            const float pq = fmaf(fmaf(w, kB3, kB2), w, kB1) * w;
            sc = (r2 > 0.0f) ? j.w * fmaf(u6, pq, v5 * cq) : 0.0f;
        } else {
            // Plummer softening: 1/(xi^2+eps^2)^(3/2), g at the unsoftened R = 2 xi
            const float x = r2 * w;
            const float c = fmaf(fmaf(fmaf(x, kA0, kA1), x, kA2), x, kA3);
            const float p = fmaf(fmaf(x, kB1, kB2), x, kB3);
            const float rs = rsqrtf(r2 + eps2);
            sc = (r2 > 0.0f) ? (j.w * fmaf(u6, p, v5 * c)) * (rs * rs * rs) : 0.0f;
        }
        ax[s] = fmaf(sc, dx, ax[s]);
        ay[s] = fmaf(sc, dy, ay[s]);
        az[s] = fmaf(sc, dz, az[s]);
    }
}

// ------------------------------------------------------------------ second-order terms
// Quadrupole part of the force of an accepted node (Sec. 4.1), added by extra passes over
// each group's list of accepted nodes.  With the pair force m f(r) D/r, f = g(R)/r^2, and
// R, r, D in eta units, the second-order Taylor term of a node with second moments Q
// about its COM is
//   B (Q D + tr(Q)/2 D) + (C/2) (D.Q.D) D,   B = g'/R^4 - 3 g/R^5,  C = g''/R^5 - 7 g'/R^6 + 15 g/R^7.
// From the factored form of Eq. 2 (g = v^5 C3(R) + u^6 P2(R), v = sat(1 - R/2), u = sat(1 - R)):
//   B R^5 = v^4 F(R) + u^5 G(R),   (C/2) R^7 = v^3 H(R) + u^4 K(R),
// with F, G, H, K the polynomials below (exact rationals; F(0)+G(0) = -3 and H(0)+K(0) =
// 15/2 give the Newtonian quadrupole).  59 FP32 operations and one rsqrt per pair, scalar:
// the constants stay immediates, and packed instructions would not save FP32-pipe cycles.
// An entry is three float4: (x, y, z, M), (Qxx, Qyy, Qzz, Qxy), (Qxz, Qyz, tr(Q)/2, 0).
__device__ __forceinline__ void quad_pair(float dx, float dy, float dz, const float4 q0, const float4 q1, float &ax,
                                          float &ay, float &az)
{
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rinv = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    const float R = r2 * rinv;
    const float v = fma_sat(R, -0.5f, 1.0f), u = add_sat(1.0f, -R);
    const float v2 = v * v, v3 = v2 * v, v4 = v2 * v2;
    const float u2 = u * u, u4 = u2 * u2, u5 = u4 * u;
    const float F = fmaf(fmaf(fmaf(fmaf(R, -4.0f, -10.057142857142857f), R, -8.457142857142857f), R,
                              -5.485714285714286f), R, -2.742857142857143f);
    const float G = fmaf(fmaf(fmaf(R, -1.0f, -2.257142857142857f), R, -1.2857142857142858f), R, -0.2571428571428571f);
    const float H = fmaf(fmaf(fmaf(fmaf(fmaf(R, 3.0f, 7.0285714285714285f), R, 12.17142857142857f), R,
                                   12.685714285714285f), R, 10.285714285714286f), R, 6.857142857142857f);
    const float K = fmaf(fmaf(fmaf(fmaf(R, 1.5f, 3.257142857142857f), R, 4.0285714285714285f), R, 2.5714285714285716f),
                         R, 0.6428571428571429f);
    const float ri2 = rinv * rinv, ri5 = ri2 * ri2 * rinv, ri7 = ri5 * ri2;
    const float B = fmaf(v4, F, u5 * G) * ri5;
    const float Ch = fmaf(v3, H, u4 * K) * ri7;
    const float qx = fmaf(q0.x, dx, fmaf(q0.w, dy, q1.x * dz));
    const float qy = fmaf(q0.w, dx, fmaf(q0.y, dy, q1.y * dz));
    const float qz = fmaf(q1.x, dx, fmaf(q1.y, dy, q0.z * dz));
    const float sd = Ch * fmaf(dx, qx, fmaf(dy, qy, dz * qz));
    ax = fmaf(B, fmaf(q1.z, dx, qx), fmaf(sd, dx, ax));
    ay = fmaf(B, fmaf(q1.z, dy, qy), fmaf(sd, dy, ay));
    az = fmaf(B, fmaf(q1.z, dz, qz), fmaf(sd, dz, az));
}

// Packed form of quad_pair for I = 2H i-particles: the same operations in the same order
// on pairs of i-particles, so each half gives quad_pair's result bit for bit; the r = 0
// select and the saturating clamps are scalar.
template <int H>
__device__ __forceinline__ void interact_quad2(const float4 j, const float4 q0, const float4 q1,
                                               const f32x2 (&xi)[H], const f32x2 (&yi)[H], const f32x2 (&zi)[H],
                                               f32x2 (&ax)[H], f32x2 (&ay)[H], f32x2 (&az)[H])
{
    const f32x2 jx = pk(j.x, j.x), jy = pk(j.y, j.y), jz = pk(j.z, j.z);
    const f32x2 qxx = pk(q0.x, q0.x), qyy = pk(q0.y, q0.y), qzz = pk(q0.z, q0.z), qxy = pk(q0.w, q0.w);
    const f32x2 qxz = pk(q1.x, q1.x), qyz = pk(q1.y, q1.y), qtr = pk(q1.z, q1.z);
    auto c2 = [](float c) { return pk(c, c); };
#pragma unroll
    for (int h = 0; h < H; h++) {
        const f32x2 dx = sub2(jx, xi[h]), dy = sub2(jy, yi[h]), dz = sub2(jz, zi[h]);
        const f32x2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
        float rl, rh;
        upk(r2, rl, rh);
        const f32x2 rinv = pk(rl > 0.0f ? rsqrtf(rl) : 0.0f, rh > 0.0f ? rsqrtf(rh) : 0.0f);
        const f32x2 R = mul2(r2, rinv);
        float Rl, Rh;
        upk(R, Rl, Rh);
        const f32x2 v = pk(fma_sat(Rl, -0.5f, 1.0f), fma_sat(Rh, -0.5f, 1.0f));
        const f32x2 u = pk(add_sat(1.0f, -Rl), add_sat(1.0f, -Rh));
        const f32x2 v2 = mul2(v, v), v3 = mul2(v2, v), v4 = mul2(v2, v2);
        const f32x2 u2 = mul2(u, u), u4 = mul2(u2, u2), u5 = mul2(u4, u);
        const f32x2 F = fma2(fma2(fma2(fma2(R, c2(-4.0f), c2(-10.057142857142857f)), R, c2(-8.457142857142857f)), R,
                                  c2(-5.485714285714286f)),
                             R, c2(-2.742857142857143f));
        const f32x2 G = fma2(fma2(fma2(R, c2(-1.0f), c2(-2.257142857142857f)), R, c2(-1.2857142857142858f)), R,
                             c2(-0.2571428571428571f));
        const f32x2 Hp = fma2(fma2(fma2(fma2(fma2(R, c2(3.0f), c2(7.0285714285714285f)), R, c2(12.17142857142857f)), R,
                                        c2(12.685714285714285f)),
                                   R, c2(10.285714285714286f)),
                              R, c2(6.857142857142857f));
        const f32x2 K = fma2(fma2(fma2(fma2(R, c2(1.5f), c2(3.257142857142857f)), R, c2(4.0285714285714285f)), R,
                                  c2(2.5714285714285716f)),
                             R, c2(0.6428571428571429f));
        const f32x2 ri2 = mul2(rinv, rinv), ri5 = mul2(mul2(ri2, ri2), rinv), ri7 = mul2(ri5, ri2);
        const f32x2 B = mul2(fma2(v4, F, mul2(u5, G)), ri5);
        const f32x2 Ch = mul2(fma2(v3, Hp, mul2(u4, K)), ri7);
        const f32x2 qx = fma2(qxx, dx, fma2(qxy, dy, mul2(qxz, dz)));
        const f32x2 qy = fma2(qxy, dx, fma2(qyy, dy, mul2(qyz, dz)));
        const f32x2 qz = fma2(qxz, dx, fma2(qyz, dy, mul2(qzz, dz)));
        const f32x2 sd = mul2(Ch, fma2(dx, qx, fma2(dy, qy, mul2(dz, qz))));
        ax[h] = fma2(B, fma2(qtr, dx, qx), fma2(sd, dx, ax[h]));
        ay[h] = fma2(B, fma2(qtr, dy, qy), fma2(sd, dy, ay[h]));
        az[h] = fma2(B, fma2(qtr, dz, qz), fma2(sd, dz, az[h]));
    }
}

template <int I>
__device__ __forceinline__ void interact_quad(const float4 j, const float4 q0, const float4 q1, const float (&xi)[I],
                                              const float (&yi)[I], const float (&zi)[I], float (&ax)[I],
                                              float (&ay)[I], float (&az)[I])
{
#pragma unroll
    for (int s = 0; s < I; s++) quad_pair(j.x - xi[s], j.y - yi[s], j.z - zi[s], q0, q1, ax[s], ay[s], az[s]);
}

// Lane layout of one pass: S parts of li = 32/S lanes, I i-particles per lane; the pass
// covers li*I of the group's remaining particles.  Cost model of a pass over a list of
// len entries, in warp cycles: each lane takes len/S entries at I*w + o cycles each (w =
// cycles per pair: packed path for even I, scalar path for odd I; o = the entry's load
// and loop overhead), the list streams through shared memory once per pass (cs cycles
// per entry), and the S parts are summed by 3*I*log2(S) shuffle-adds (cr cycles each).
// For n <= 32*kImax remaining particles the first pass of the cheapest sequence of
// passes covering n (at a typical list length) is tabulated at compile time by dynamic
// programming over n; larger groups take the widest layout (S = 1, I = kImax).
#ifndef GREEM_LAYOUT_W_EVEN
#define GREEM_LAYOUT_W_EVEN 29
#endif
#ifndef GREEM_LAYOUT_W_ODD
#define GREEM_LAYOUT_W_ODD 39
#endif
#ifndef GREEM_LAYOUT_O
#define GREEM_LAYOUT_O 8
#endif
#ifndef GREEM_LAYOUT_CS
#define GREEM_LAYOUT_CS 2
#endif
struct LayoutTable {
    uint8_t v[32 * kImax + 1];  // log2(S) in bits 4-6, I in bits 0-3
};

constexpr LayoutTable make_layout_table()
{
    constexpr long len = 512, cr = 3;
    LayoutTable t{};
    long cost[32 * kImax + 1] = {};
    for (int n = 1; n <= 32 * kImax; n++) {
        long best = -1;
        for (int ls = 5; ls >= 0; ls--) {      // more parts first: they win ties
            const int li = 32 >> ls;
            for (int I = 1; I <= kImax; I++) {
                const long w = (I % 2 == 0) ? GREEM_LAYOUT_W_EVEN : GREEM_LAYOUT_W_ODD;
                const int rest = n - li * I;
                const long pass = (len * li * (I * w + GREEM_LAYOUT_O)) / 32 +
                                  len * GREEM_LAYOUT_CS + 3L * I * ls * cr;
                const long c = pass + cost[rest > 0 ? rest : 0];
                if (best < 0 || c < best) {
                    best = c;
                    t.v[n] = (uint8_t)((ls << 4) | I);
                }
            }
        }
        cost[n] = best;
    }
    return t;
}

__constant__ LayoutTable c_layout = make_layout_table();

__device__ __forceinline__ void choose_layout(uint32_t n, int &S, int &I)
{
    if (n > 32u * kImax) {
        S = 1;
        I = kImax;
        return;
    }
    const uint32_t v = c_layout.v[n];
    S = 1 << (v >> 4);
    I = (int)(v & 15u);
}

// Layout of a second-order pass: I in {1, 2, 4} only (the pair body is long, and fewer
// instantiations keep the instruction cache warm), the fewest slots li*I >= n (ties: more
// parts); when that wastes more than n/4 slots and n > 32, the largest slot count <= n.
__device__ __forceinline__ void choose_layout_quad(uint32_t n, int &S, int &I)
{
    if (n >= 128u) {
        S = 1;
        I = 4;
        return;
    }
    int bs = 1, bi = 4;
    uint32_t best = 0xffffffffu;
#pragma unroll
    for (int s = 32; s >= 1; s >>= 1) {
#pragma unroll
        for (int i = 1; i <= 4; i <<= 1) {
            const uint32_t slots = (32u / s) * (uint32_t)i;
            if (slots >= n && slots < best) {
                best = slots;
                bs = s;
                bi = i;
            }
        }
    }
    if (n > 32u && best - n > n / 4u) {
        uint32_t lo = 0;
#pragma unroll
        for (int s = 32; s >= 1; s >>= 1) {
#pragma unroll
            for (int i = 1; i <= 4; i <<= 1) {
                const uint32_t slots = (32u / s) * (uint32_t)i;
                if (slots <= n && slots > lo) {
                    lo = slots;
                    bs = s;
                    bi = i;
                }
            }
        }
    }
    S = bs;
    I = bi;
}

struct WarpPipe {
    float4 *buf[2];
    uint64_t *bar;
    uint32_t ph[2];
};

// Stages entries [c*ce, min((c+1)*ce, len)) of a list (stride float4 per entry, starting
// at float4 lo of src) into buffer b.
__device__ __forceinline__ void issue_chunk(const float4 *src, uint32_t ce, uint32_t stride, WarpPipe &wp, int b,
                                            unsigned long long lo, uint32_t c, uint32_t len, int lane)
{
    if (lane == 0) {
        const uint32_t first = c * ce;
        const uint32_t nj = min(ce, len - first);
        const uint32_t bytes = nj * stride * (uint32_t)sizeof(float4);
        fence_proxy_async();
        mbar_arrive_tx(&wp.bar[b], bytes);
        bulk_g2s(wp.buf[b], src + lo + (unsigned long long)first * stride, bytes, &wp.bar[b]);
    }
}

// One pass of a group: I i-particles per lane, S parts; returns false on a timeout.  QUAD:
// the pass runs over the group's accepted nodes (three float4 per entry) and adds their
// second-order terms to the accelerations the monopole passes stored.
template <int I, bool SOFT, bool QUAD>
__device__ __noinline__ bool group_pass(const ForceArgs &a, const Group &gr, uint32_t done, int S,
                                        unsigned long long lo, uint32_t len, WarpPipe &wp, float scale, float eps2,
                                        int lane)
{
    const unsigned FULL = 0xffffffffu;
    const int li = 32 / S;
    const int slot = lane & (li - 1);
    const int part = lane / li;
    const uint32_t gend = gr.begin + gr.count;
    float xi[I], yi[I], zi[I], ax[I], ay[I], az[I];
#pragma unroll
    for (int s = 0; s < I; s++) {
        const uint32_t idx = gr.begin + done + (uint32_t)(s * li + slot);
        float4 v = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.f);
        if (idx < gend) v = a.irel[idx];
        // the second-order terms work in eta = r_cut/2 units (exact rescaling)
        xi[s] = QUAD ? 2.0f * v.x : v.x;
        yi[s] = QUAD ? 2.0f * v.y : v.y;
        zi[s] = QUAD ? 2.0f * v.z : v.z;
        ax[s] = ay[s] = az[s] = 0.f;
    }
    constexpr bool kPacked = (I % 2) == 0;
    constexpr uint32_t stride = QUAD ? 3u : 1u;
    const uint32_t ce = QUAD ? (uint32_t)a.chunk / 4u : (uint32_t)a.chunk;
    const float4 *src = QUAD ? a.qlist : a.flist;
    constexpr int H = kPacked ? I / 2 : 1;
    f32x2 xi2[H], yi2[H], zi2[H], ax2[H], ay2[H], az2[H];
    const f32x2 eps2x2 = pk(eps2, eps2);
    if constexpr (kPacked) {
#pragma unroll
        for (int h = 0; h < H; h++) {
            xi2[h] = pk(xi[2 * h], xi[2 * h + 1]);
            yi2[h] = pk(yi[2 * h], yi[2 * h + 1]);
            zi2[h] = pk(zi[2 * h], zi[2 * h + 1]);
            ax2[h] = ay2[h] = az2[h] = pk(0.f, 0.f);
        }
    }
    const uint32_t nch = (len + ce - 1) / ce;
    const uint32_t polls = a.wait_polls1 ? a.wait_polls1 - 1u : kWaitPolls;
    if (nch) issue_chunk(src, ce, stride, wp, 0, lo, 0, len, lane);
    bool ok = true;
    for (uint32_t c = 0; c < nch; c++) {
        const int b = (int)(c & 1u);
        if (c + 1 < nch) issue_chunk(src, ce, stride, wp, b ^ 1, lo, c + 1, len, lane);
        const bool got = mbar_wait_bounded(&wp.bar[b], wp.ph[b], polls);
        if (!__all_sync(FULL, got)) {
            ok = false;
            // the warp leaves the kernel: let every copy it has in flight land first, the
            // chunk it gave up on and the prefetched one (at the full poll limit)
            mbar_wait_bounded(&wp.bar[b], wp.ph[b], kWaitPolls);
            if (c + 1 < nch) mbar_wait_bounded(&wp.bar[b ^ 1], wp.ph[b ^ 1], kWaitPolls);
            break;
        }
        wp.ph[b] ^= 1u;
        const float4 *buf = wp.buf[b];
        const uint32_t nj = min(ce, len - c * ce);
        if constexpr (QUAD && kPacked) {
#pragma unroll 1
            for (uint32_t t = (uint32_t)part; t < nj; t += (uint32_t)S)
                interact_quad2<H>(buf[3 * t], buf[3 * t + 1], buf[3 * t + 2], xi2, yi2, zi2, ax2, ay2, az2);
        } else if constexpr (QUAD) {
#pragma unroll 1
            for (uint32_t t = (uint32_t)part; t < nj; t += (uint32_t)S)
                interact_quad<I>(buf[3 * t], buf[3 * t + 1], buf[3 * t + 2], xi, yi, zi, ax, ay, az);
        } else if constexpr (kPacked) {
#pragma unroll(kUnroll)
            for (uint32_t t = (uint32_t)part; t < nj; t += (uint32_t)S) {
                const float4 j = buf[t];
                interact2<H, SOFT>(j, xi2, yi2, zi2, ax2, ay2, az2, eps2x2);
            }
        } else if constexpr (I <= 2) {
#pragma unroll 4
            for (uint32_t t = (uint32_t)part; t < nj; t += (uint32_t)S) {
                const float4 j = buf[t];
                interact<I, SOFT>(j, xi, yi, zi, ax, ay, az, eps2);
            }
        } else {
#pragma unroll(kUnroll)
            for (uint32_t t = (uint32_t)part; t < nj; t += (uint32_t)S) {
                const float4 j = buf[t];
                interact<I, SOFT>(j, xi, yi, zi, ax, ay, az, eps2);
            }
        }
        __syncwarp();
    }
    if constexpr (kPacked) {
#pragma unroll
        for (int h = 0; h < H; h++) {
            upk(ax2[h], ax[2 * h], ax[2 * h + 1]);
            upk(ay2[h], ay[2 * h], ay[2 * h + 1]);
            upk(az2[h], az[2 * h], az[2 * h + 1]);
        }
    }
#pragma unroll
    for (int s = 0; s < I; s++) {
        for (int o = li; o < 32; o <<= 1) {
            ax[s] += __shfl_xor_sync(FULL, ax[s], o);
            ay[s] += __shfl_xor_sync(FULL, ay[s], o);
            az[s] += __shfl_xor_sync(FULL, az[s], o);
        }
    }
    if (part == 0) {
        float *acc = static_cast<float *>(a.acc);
#pragma unroll
        for (int s = 0; s < I; s++) {
            const uint32_t idx = gr.begin + done + (uint32_t)(s * li + slot);
            if (idx < gend) {
                const size_t p = (size_t)a.perm[idx] * 3;
                if (QUAD) {
                    acc[p] += ax[s] * scale;
                    acc[p + 1] += ay[s] * scale;
                    acc[p + 2] += az[s] * scale;
                } else {
                    acc[p] = ax[s] * scale;
                    acc[p + 1] = ay[s] * scale;
                    acc[p + 2] = az[s] * scale;
                }
            }
        }
    }
    return ok;
}

// QUAD: the second-order passes over the groups' accepted nodes (after the monopole
// launch; groups without accepted nodes are skipped).
template <bool SOFT, bool QUAD>
__global__ void __launch_bounds__(GREEM_FORCE_THREADS, GREEM_FORCE_MINB) k_force_f32(ForceArgs a)
{
    extern __shared__ __align__(128) float4 sm[];
    __shared__ __align__(8) uint64_t bars[16][2];
    const unsigned FULL = 0xffffffffu;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpPipe wp;
    wp.buf[0] = sm + (size_t)w * 2 * a.chunk;
    wp.buf[1] = wp.buf[0] + a.chunk;
    wp.bar = bars[w];
    wp.ph[0] = wp.ph[1] = 0;
    if (lane == 0) {
        mbar_init(&wp.bar[0], 1);
        mbar_init(&wp.bar[1], 1);
        fence_barrier_init();
    }
    __syncwarp();
    if (a.st->flags & ST_NODE_CAP) return;  // the tree was truncated: the call is retried
    // the quadrupole lists are incomplete (and would be read past their end): the call is
    // retried with larger lists
    if (QUAD && (a.st->flags & (ST_LIST_CAP | ST_QLIST_CAP))) return;
    const uint32_t G = *a.n_groups;
    for (;;) {
        unsigned long long gi = 0;
        if (lane == 0) gi = atomicAdd(&a.st->work[QUAD ? 3 : 1], 1ull);
        gi = __shfl_sync(FULL, gi, 0);
        if (gi >= G) break;
        const uint32_t g = a.order ? a.order[gi] : (uint32_t)gi;
        const Group gr = a.groups[g];
        const BoxPar &bp = a.bps[gr.box];
        // r_cut-unit accelerations (eta-unit ones in the second-order passes) -> physical
        const float scale = QUAD ? 4.0f * bp.inv_rc2 : bp.inv_rc2, eps2 = bp.eps2;
        const unsigned long long lo = QUAD ? 3ull * a.qoff[g] : a.loff[g];
        const uint32_t len = QUAD ? a.qcnt[g] : a.llen[g];
        if (QUAD && len == 0) continue;
        uint32_t done = 0;
        unsigned long long evals = 0;
        bool ok = true;
        while (done < gr.count && ok) {
            int S, I;
            if (QUAD) {
                choose_layout_quad(gr.count - done, S, I);
                if (I == 1) ok = group_pass<1, SOFT, true>(a, gr, done, S, lo, len, wp, scale, eps2, lane);
                else if (I == 2) ok = group_pass<2, SOFT, true>(a, gr, done, S, lo, len, wp, scale, eps2, lane);
                else ok = group_pass<4, SOFT, true>(a, gr, done, S, lo, len, wp, scale, eps2, lane);
                done += (uint32_t)(32 / S) * (uint32_t)I;
                continue;
            }
            choose_layout(gr.count - done, S, I);
            switch (I) {
            case 1: ok = group_pass<1, SOFT, false>(a, gr, done, S, lo, len, wp, scale, eps2, lane); break;
            case 2: ok = group_pass<2, SOFT, false>(a, gr, done, S, lo, len, wp, scale, eps2, lane); break;
            case 3: ok = group_pass<3, SOFT, false>(a, gr, done, S, lo, len, wp, scale, eps2, lane); break;
            case 4: ok = group_pass<4, SOFT, false>(a, gr, done, S, lo, len, wp, scale, eps2, lane); break;
#if GREEM_FORCE_IMAX >= 5
            case 5: ok = group_pass<5, SOFT, false>(a, gr, done, S, lo, len, wp, scale, eps2, lane); break;
#endif
#if GREEM_FORCE_IMAX >= 6
            case 6: ok = group_pass<6, SOFT, false>(a, gr, done, S, lo, len, wp, scale, eps2, lane); break;
#endif
#if GREEM_FORCE_IMAX >= 7
            case 7: ok = group_pass<7, SOFT, false>(a, gr, done, S, lo, len, wp, scale, eps2, lane); break;
#endif
#if GREEM_FORCE_IMAX >= 8
            case 8: ok = group_pass<8, SOFT, false>(a, gr, done, S, lo, len, wp, scale, eps2, lane); break;
#endif
            default: ok = false; break;  // not reachable: choose_layout never exceeds kImax
            }
            const uint32_t slots = (uint32_t)(32 / S) * (uint32_t)I;
            evals += (unsigned long long)slots * len;
            done += slots;
        }
        if (!QUAD && lane == 0) atomicAdd(&a.st->sum_eval, evals);
        if (!ok) {
            if (lane == 0) atomicOr(&a.st->flags, ST_TIMEOUT);
            break;
        }
    }
}

// The accepted nodes of each group's list, compacted in list order into the group's
// stretch [qoff[g], qoff[g] + qcnt[g]) of the quadrupole list (three float4 per entry:
// the list entry, then the node's second moments, both in eta units).  One warp per group.  An overflow of
// qcap entries records the total needed and the call is retried with a larger list.
__global__ void __launch_bounds__(256) k_qlist_fill(ForceArgs a, const float4 *__restrict__ quad, unsigned long long qcap)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (a.st->flags & (ST_NODE_CAP | ST_LIST_CAP)) return;
    const uint32_t G = *a.n_groups;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long need = a.qoff[G];
        if (need > qcap) {
            a.st->sum_quad = need;
            atomicOr(&a.st->flags, ST_QLIST_CAP);
        }
    }
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
        const unsigned long long lo = a.loff[g];
        const uint32_t len = a.lraw[g];
        const unsigned long long q0 = a.qoff[g];
        if (q0 + a.qcnt[g] > qcap) continue;
        uint32_t k = 0;
        for (uint32_t e0 = 0; e0 < len; e0 += 32) {
            const uint32_t e = e0 + lane;
            unsigned long long ie = 0;
            if (e < len) ie = a.ilist[lo + e];
            const bool node = e < len && ((ie >> 32) & 1ull) != 0;
            const unsigned bal = __ballot_sync(FULL, node);
            if (node) {
                const uint32_t n = (uint32_t)(ie & 0xffffffffull);
                float4 *d = const_cast<float4 *>(a.qlist) + 3ull * (q0 + k + __popc(bal & lt));
                // r_cut units -> eta units (positions x2, second moments x4; exact)
                const float4 f = a.flist[lo + e], q0 = quad[2 * (size_t)n], q1 = quad[2 * (size_t)n + 1];
                d[0] = make_float4(2.0f * f.x, 2.0f * f.y, 2.0f * f.z, f.w);
                d[1] = make_float4(4.0f * q0.x, 4.0f * q0.y, 4.0f * q0.z, 4.0f * q0.w);
                d[2] = make_float4(4.0f * q1.x, 4.0f * q1.y, 4.0f * q1.z, 4.0f * q1.w);
            }
            k += __popc(bal);
        }
    }
}

void launch_qlist_fill(const ForceArgs &a, const float4 *quad, unsigned long long qcap, cudaStream_t s, int nsm)
{
    k_qlist_fill<<<nsm * 8, 256, 0, s>>>(a, quad, qcap);
    g_launches++;
}

// ------------------------------------------------------------------ work order
// Groups are ordered by lane layout (I i-particles per lane, S parts), largest first, so
// that the warps of an SM mostly run the same instantiation of group_pass at a time
// (one instruction-cache footprint) and the cheapest groups come last.
__device__ __forceinline__ int layout_bin(uint32_t n)
{
    if (n > 32u * kImax) return 0;
    int S, I;
    choose_layout(n, S, I);
    return (8 - I) * 6 + (31 - __clz(S));
}

__global__ void __launch_bounds__(256) k_bin_count(const Group *__restrict__ groups, const uint32_t *n_groups,
                                                   uint32_t *__restrict__ bins)
{
    __shared__ uint32_t sb[64];
    if (threadIdx.x < 64) sb[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t G = *n_groups;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
        atomicAdd(&sb[layout_bin(groups[g].count)], 1u);
    __syncthreads();
    if (threadIdx.x < 64 && sb[threadIdx.x]) atomicAdd(&bins[threadIdx.x], sb[threadIdx.x]);
}

__global__ void k_bin_scan(uint32_t *bins)
{
    const uint32_t lane = threadIdx.x;
    const uint32_t v0 = bins[lane], v1 = bins[32 + lane];
    uint32_t x0 = v0, x1 = v1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, x1, o);
        if (lane >= (uint32_t)o) {
            x0 += y0;
            x1 += y1;
        }
    }
    const uint32_t tot0 = __shfl_sync(0xffffffffu, x0, 31);
    bins[64 + lane] = x0 - v0;        // cursors
    bins[96 + lane] = tot0 + x1 - v1;
}

__global__ void __launch_bounds__(256) k_bin_scatter(const Group *__restrict__ groups, const uint32_t *n_groups,
                                                     uint32_t *__restrict__ bins, uint32_t *__restrict__ order)
{
    const uint32_t G = *n_groups;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    // whole warps iterate together so that the bin atomics can be aggregated per warp
    for (uint32_t g0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); g0 < G; g0 += stride) {
        const uint32_t g = g0 + lane;
        const uint32_t key = g < G ? (uint32_t)layout_bin(groups[g].count) : 1024u;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (g < G && lane == leader) base = atomicAdd(&bins[64 + key], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (g < G) order[base + __popc(peers & ((1u << lane) - 1u))] = g;
    }
}

void launch_force_order(const Group *groups, const uint32_t *n_groups, uint32_t *bins, uint32_t *order,
                        cudaStream_t s, int nsm)
{
    cudaMemsetAsync(bins, 0, 128 * sizeof(uint32_t), s);
    k_bin_count<<<nsm * 4, 256, 0, s>>>(groups, n_groups, bins);
    k_bin_scan<<<1, 32, 0, s>>>(bins);
    k_bin_scatter<<<nsm * 4, 256, 0, s>>>(groups, n_groups, bins, order);
    g_launches += 3;
}

// Per device: the shared-memory opt-in of each force-kernel instantiation, and its
// occupancy per block shape as (smem << 8) | blocks per SM (0 = not queried yet).
struct ForceLaunchCache {
    std::atomic<int> smem_set[3];
    std::atomic<long long> occ[3][17];
};
static ForceLaunchCache g_force_cache[kMaxDevices];

// Dynamic shared memory of the FP32 force kernel: two chunk buffers per warp.
size_t force_smem_bytes(int chunk, int warps)
{
    return (size_t)warps * 2 * (size_t)chunk * sizeof(float4);
}

void launch_force_f32(const ForceArgs &a, cudaStream_t s, int nsm, bool soft, bool quad)
{
    const int threads = 32 * a.warps;
    const size_t smem = force_smem_bytes(a.chunk, a.warps);
    auto kern = quad ? k_force_f32<false, true> : (soft ? k_force_f32<true, false> : k_force_f32<false, false>);
    const int which = quad ? 2 : (soft ? 1 : 0);
    // the opt-in applies to the current device only; the occupancy is queried once per
    // device and shape (not while a stream is being captured)
    const int dev = current_device_index();
    ForceLaunchCache *fc = dev >= 0 ? &g_force_cache[dev] : nullptr;
    if (!fc || fc->smem_set[which].load() < (int)smem) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kForceSmemMax);
        if (fc) fc->smem_set[which].store((int)kForceSmemMax);
    }
    const long long key = (long long)smem << 8;
    long long occ = fc ? fc->occ[which][a.warps].load() : 0;
    if ((occ & ~0xffll) != key || (occ & 0xff) == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        per_sm = per_sm < 1 ? 1 : (per_sm > 255 ? 255 : per_sm);
        occ = key | per_sm;
        if (fc) fc->occ[which][a.warps].store(occ);
    }
    const int per_sm = (int)(occ & 0xff);
    kern<<<nsm * per_sm, threads, smem, s>>>(a);
    g_launches++;
}

// ------------------------------------------------------------------ FP64 form
// The same lists as index entries; absolute FP64 positions of particles and node
// centres of mass, the entry's image shift, and Eq. 1-2 in FP64.  It is the plain form
// the FP32 kernel is compared with.
template <int I>
__device__ __noinline__ void group_pass_f64(const ForceArgs &a, const Group &gr, const BoxPar &bp, uint32_t done,
                                            int S, unsigned long long lo, uint32_t len, Dbl4 *jb, int lane)
{
    const unsigned FULL = 0xffffffffu;
    const int li = 32 / S;
    const int slot = lane & (li - 1);
    const int part = lane / li;
    const uint32_t gend = gr.begin + gr.count;
    const double L = bp.L, ie = bp.inv_eta, eps2 = bp.eps * bp.eps;
    double xi[I], yi[I], zi[I], ax[I], ay[I], az[I];
#pragma unroll
    for (int s = 0; s < I; s++) {
        const uint32_t idx = gr.begin + done + (uint32_t)(s * li + slot);
        const bool v = idx < gend;
        xi[s] = v ? a.xs[idx] : 1.0e30;
        yi[s] = v ? a.ys[idx] : 1.0e30;
        zi[s] = v ? a.zs[idx] : 1.0e30;
        ax[s] = ay[s] = az[s] = 0.0;
    }
    for (uint32_t c = 0; c < len; c += 32) {
        const uint32_t e = c + (uint32_t)lane;
        Dbl4 jv = make_dbl4(1.0e30, 1.0e30, 1.0e30, 0.0);
        if (e < len) {
            const unsigned long long en = a.ilist[lo + e];
            const uint32_t idx = (uint32_t)en;
            const unsigned code = (unsigned)(en >> 33) & 63u;
            auto sh = [L](unsigned c2) { return c2 == 1u ? L : (c2 == 2u ? -L : 0.0); };
            if (en & (1ull << 32)) {
                const Dbl4 mm = a.mom64[idx];
                jv = make_dbl4(mm.x + sh(code & 3u), mm.y + sh((code >> 2) & 3u), mm.z + sh((code >> 4) & 3u), mm.w);
            } else {
                jv = make_dbl4(a.xs[idx] + sh(code & 3u), a.ys[idx] + sh((code >> 2) & 3u),
                                  a.zs[idx] + sh((code >> 4) & 3u), (double)a.ms[idx]);
            }
        }
        jb[lane] = jv;
        __syncwarp();
        const uint32_t nj = min(32u, len - c);
        for (uint32_t t = (uint32_t)part; t < nj; t += (uint32_t)S) {
            const Dbl4 j = jb[t];
#pragma unroll
            for (int s = 0; s < I; s++) {
                const double dx = j.x - xi[s], dy = j.y - yi[s], dz = j.z - zi[s];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 > 0.0) {
                    const double rinv = rsqrt(r2);
                    const double R = r2 * rinv * ie;
                    if (R < 2.0) {
                        const double v = 1.0 - 0.5 * R;
                        const double u = R < 1.0 ? 1.0 - R : 0.0;
                        const double v2 = v * v, u2 = u * u;
                        const double g = v2 * v2 * v * (8.0 / 35.0) * (((7.0 * R + 22.0) * R + 10.0) * R + 4.0) +
                                         u2 * u2 * u2 * ((7.0 * R + 18.0) * R + 3.0) / 35.0;
                        double rinv3;
                        if (eps2 > 0.0) {
                            const double rs = rsqrt(r2 + eps2);
                            rinv3 = rs * rs * rs;
                        } else {
                            rinv3 = rinv * rinv * rinv;
                        }
                        const double f = j.w * g * rinv3;
                        ax[s] += f * dx;
                        ay[s] += f * dy;
                        az[s] += f * dz;
                    }
                }
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int s = 0; s < I; s++) {
        for (int o = li; o < 32; o <<= 1) {
            ax[s] += __shfl_xor_sync(FULL, ax[s], o);
            ay[s] += __shfl_xor_sync(FULL, ay[s], o);
            az[s] += __shfl_xor_sync(FULL, az[s], o);
        }
    }
    if (part == 0) {
        double *acc = static_cast<double *>(a.acc);
#pragma unroll
        for (int s = 0; s < I; s++) {
            const uint32_t idx = gr.begin + done + (uint32_t)(s * li + slot);
            if (idx < gend) {
                const size_t p = (size_t)a.perm[idx] * 3;
                acc[p] = ax[s];
                acc[p + 1] = ay[s];
                acc[p + 2] = az[s];
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_force_f64(ForceArgs a)
{
    __shared__ Dbl4 jbuf[8][32];
    const unsigned FULL = 0xffffffffu;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (a.st->flags & ST_NODE_CAP) return;
    const uint32_t G = *a.n_groups;
    for (;;) {
        unsigned long long gi = 0;
        if (lane == 0) gi = atomicAdd(&a.st->work[2], 1ull);
        gi = __shfl_sync(FULL, gi, 0);
        if (gi >= G) break;
        const uint32_t g = a.order ? a.order[gi] : (uint32_t)gi;
        const Group gr = a.groups[g];
        const BoxPar &bp = a.bps[gr.box];
        const unsigned long long lo = a.loff[g];
        const uint32_t len = a.lraw[g];
        uint32_t done = 0;
        unsigned long long evals = 0;
        while (done < gr.count) {
            int S, I;
            choose_layout(gr.count - done, S, I);
            switch (I) {
            case 1: group_pass_f64<1>(a, gr, bp, done, S, lo, len, jbuf[w], lane); break;
            case 2: group_pass_f64<2>(a, gr, bp, done, S, lo, len, jbuf[w], lane); break;
            case 3: group_pass_f64<3>(a, gr, bp, done, S, lo, len, jbuf[w], lane); break;
            case 4: group_pass_f64<4>(a, gr, bp, done, S, lo, len, jbuf[w], lane); break;
            case 5: group_pass_f64<5>(a, gr, bp, done, S, lo, len, jbuf[w], lane); break;
            case 6: group_pass_f64<6>(a, gr, bp, done, S, lo, len, jbuf[w], lane); break;
            case 7: group_pass_f64<7>(a, gr, bp, done, S, lo, len, jbuf[w], lane); break;
            default: group_pass_f64<8>(a, gr, bp, done, S, lo, len, jbuf[w], lane); break;
            }
            const uint32_t slots = (uint32_t)(32 / S) * (uint32_t)I;
            evals += (unsigned long long)slots * len;
            done += slots;
        }
        if (lane == 0) atomicAdd(&a.st->sum_eval, evals);
    }
}

void launch_force_f64(const ForceArgs &a, cudaStream_t s, int nsm)
{
    static std::atomic<int> cached[kMaxDevices];
    const int dev = current_device_index();
    int per_sm = dev >= 0 ? cached[dev].load() : 0;
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_f64, 256, 0);
        if (per_sm < 1) per_sm = 1;
        if (dev >= 0) cached[dev].store(per_sm);
    }
    k_force_f64<<<nsm * per_sm, 256, 0, s>>>(a);
    g_launches++;
}

// ------------------------------------------------------------------ pairwise experiment
// Every pair k becomes a one-particle group with a one-entry list (padded to 8):
// i and j are passed relative to x_g in r_cut units (FP64 subtract, one FP32 rounding).
__global__ void k_pair_setup(const double *__restrict__ xg, const double *__restrict__ xi,
                             const double *__restrict__ xj, const float *__restrict__ mj, uint32_t np, double inv_rc,
                             Group *groups, float4 *irel, float4 *flist, unsigned long long *loff, uint32_t *llen,
                             uint32_t *lraw, uint32_t *perm, uint32_t *n_groups)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) *n_groups = np;
    if (k >= np) return;
    Group g;
    g.node = 0;
    g.begin = k;
    g.count = 1;
    g.box = 0;
    g.cx = g.cy = g.cz = 0;
    g.hg = 0;
    groups[k] = g;
    float r[3], q[3];
    for (int c = 0; c < 3; c++) {
        r[c] = (float)__dmul_rn(__dsub_rn(xi[3 * (size_t)k + c], xg[3 * (size_t)k + c]), inv_rc);
        q[c] = (float)__dmul_rn(__dsub_rn(xj[3 * (size_t)k + c], xg[3 * (size_t)k + c]), inv_rc);
    }
    irel[k] = make_float4(r[0], r[1], r[2], 0.f);
    flist[8 * (size_t)k] = make_float4(q[0], q[1], q[2], mj[k]);
    for (int e = 1; e < 8; e++) flist[8 * (size_t)k + e] = make_float4(16.f, 16.f, 16.f, 0.f);
    loff[k] = 8ull * k;
    llen[k] = 8;
    lraw[k] = 1;
    perm[k] = k;
}

void launch_pair_setup(const double *xg, const double *xi, const double *xj, const float *mj, uint32_t np,
                       double inv_rc, Group *groups, float4 *irel, float4 *flist, unsigned long long *loff,
                       uint32_t *llen, uint32_t *lraw, uint32_t *perm, uint32_t *n_groups, cudaStream_t s)
{
    k_pair_setup<<<(np + 255) / 256, 256, 0, s>>>(xg, xi, xj, mj, np, inv_rc, groups, irel, flist, loff, llen, lraw,
                                                   perm, n_groups);
    g_launches++;
}

// ------------------------------------------------------------------ peak microbenchmarks
__global__ void __launch_bounds__(256) k_peak_f32(float *out, int iters)
{
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = threadIdx.x * 1e-9f + k;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = fmaf(v[k], 0.9999f, 1e-7f);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += v[k];
    if (s == 1234.5f) out[0] = s;
}

__global__ void __launch_bounds__(256) k_peak_f64(double *out, int iters)
{
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = threadIdx.x * 1e-9 + k;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] = fma(v[k], 0.9999, 1e-7);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += v[k];
    if (s == 1234.5) out[0] = s;
}

// The force kernel's own packed pair loop (interact2, six i-particles per lane) over 256
// list entries held in shared memory, with no list streaming and no group overhead: the
// rate this formulation reaches by itself, counted at 42 flops per pair.
__global__ void __launch_bounds__(256) k_peak_pairloop(float *out, int iters)
{
    __shared__ float4 sj[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        sj[t] = make_float4(0.3f + t * 1e-3f, 0.2f - t * 1e-3f, 0.1f + t * 2e-3f, 1e-3f);
    __syncthreads();
    constexpr int H = 3;
    f32x2 xi[H], yi[H], zi[H], ax[H], ay[H], az[H];
#pragma unroll
    for (int h = 0; h < H; h++) {
        const float b = threadIdx.x * 1e-4f + h * 0.01f;
        xi[h] = pk(b, b + 1e-3f);
        yi[h] = pk(0.5f * b, b);
        zi[h] = pk(b, -b);
        ax[h] = ay[h] = az[h] = pk(0.f, 0.f);
    }
    const f32x2 eps2 = pk(0.f, 0.f);
    for (int it = 0; it < iters; it++) {
#pragma unroll(kUnroll)
        for (int t = 0; t < 256; t++) interact2<H, false>(sj[t], xi, yi, zi, ax, ay, az, eps2);
    }
    float sum = 0.f;
#pragma unroll
    for (int h = 0; h < H; h++) {
        float a, b;
        upk(ax[h], a, b);
        sum += a + b;
        upk(ay[h], a, b);
        sum += a + b;
        upk(az[h], a, b);
        sum += a + b;
    }
    if (sum == 1234.5f) out[0] = sum;
}

double peak_tflops(int which, int nsm, cudaStream_t s, int *err)
{
    *err = 0;
    void *out = nullptr;
    if (cudaMalloc(&out, 64) != cudaSuccess) {
        *err = -3;
        return 0.0;
    }
    const int blocks = which == 2 ? nsm * 2 : nsm * 8, threads = 256;
    const int iters = which == 0 ? 4000 : (which == 1 ? 64 : 40);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0, s);
        if (which == 0) k_peak_f32<<<blocks, threads, 0, s>>>((float *)out, iters);
        else if (which == 1) k_peak_f64<<<blocks, threads, 0, s>>>((double *)out, iters);
        else k_peak_pairloop<<<blocks, threads, 0, s>>>((float *)out, iters);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = which == 2 ? 42.0 * 6 * 256 * (double)iters * blocks * threads
                                        : 2.0 * 8 * 16 * (double)iters * blocks * threads;
        const double tf = flops / (ms * 1e-3) / 1e12;
        if (rep > 0 && tf > best) best = tf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) *err = -2;
    cudaFree(out);
    return best;
}

}  // namespace greem
