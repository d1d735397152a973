// S1 wrap + 63-bit Morton keys, S2 stable LSD radix sort and the SoA gather.
//
// Key (Sec. 3.2.5 "morton key", 12 bytes with the index): each coordinate is wrapped
// into [0, L) (periodic box), mapped to a 21-bit cell index floor((x/L) 2^21) clamped
// to 2^21-1, and the three indices are bit-interleaved with x as the high bit of each
// 3-bit digit.  Every FP64 step uses explicit round-to-nearest intrinsics so that no
// multiply-add is fused: the key is a pure function of the IEEE inputs.
#include "common.cuh"

namespace greem {

// floor((r/L) 2^21) clamped to [0, 2^21-1].  r * (1/L) differs from the rounded
// quotient by at most 3 ulp, i.e. by < 1e-9 after the scaling, so its floor is the same
// unless the scaled value lies within 1e-6 of an integer; only then is the exact
// quotient formed.
__device__ __forceinline__ uint32_t cell21(double r, double L, double invL)
{
    double q = __dmul_rn(__dmul_rn(r, invL), 2097152.0);
    double f = floor(q);
    const double fr = q - f;
    if (fr < 1e-6 || fr > 1.0 - 1e-6) f = floor(__dmul_rn(__ddiv_rn(r, L), 2097152.0));
    long long i = (long long)f;
    i = i < 0 ? 0 : i;
    i = i > 2097151 ? 2097151 : i;
    return (uint32_t)i;
}

__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

// Power-of-two box side (the usual L = 1): (r/L) 2^21 = r 2^(21-e) exactly, so the cell
// index is read from the bits of r with integer operations only (no FP64 pipe work).
// Same result as cell21(): the quotient is exact, and floor of the scaled value is the
// integer part of the binary expansion.
__device__ __forceinline__ uint32_t cell21_pow2(double r, int e)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(r);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;  // zero or subnormal
    const unsigned long long mant = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = (ex - 1023) - 52 + 21 - e;  // value = mant * 2^sh
    long long i;
    if (sh >= 0) i = sh >= 11 ? (1ll << 62) : (long long)(mant << sh);
    else i = -sh >= 64 ? 0 : (long long)(mant >> (-sh));
    i = i > 2097151 ? 2097151 : i;
    return (uint32_t)i;
}

__global__ void __launch_bounds__(256) k_keys(const double *__restrict__ pos, uint32_t N,
                                              const uint32_t *__restrict__ box_off, int nbox,
                                              const BoxPar *__restrict__ bps, uint64_t *__restrict__ keys,
                                              DevStatus *st)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const BoxPar &bp = bps[box_of(i, box_off, nbox)];
    const double L = bp.L, invL = bp.inv_L;
    double x = pos[3 * (size_t)i], y = pos[3 * (size_t)i + 1], z = pos[3 * (size_t)i + 2];
    // finite test on the exponent bits (integer pipe)
    const auto nonfinite = [](double v) {
        return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
    };
    if (nonfinite(x) || nonfinite(y) || nonfinite(z)) {
        atomicOr(&st->flags, ST_NONFINITE);
        keys[i] = 0;
        return;
    }
    uint32_t cx, cy, cz;
    if (bp.pow2_e != kNotPow2) {
        cx = cell21_pow2(wrap_pos_fast(x, L), bp.pow2_e);
        cy = cell21_pow2(wrap_pos_fast(y, L), bp.pow2_e);
        cz = cell21_pow2(wrap_pos_fast(z, L), bp.pow2_e);
    } else {
        cx = cell21(wrap_pos_fast(x, L), L, invL);
        cy = cell21(wrap_pos_fast(y, L), L, invL);
        cz = cell21(wrap_pos_fast(z, L), L, invL);
    }
    keys[i] = (spread3(cx) << 2) | (spread3(cy) << 1) | spread3(cz);
}

void launch_keys(const double *pos, uint32_t N, const uint32_t *box_off, int nbox, const BoxPar *bps,
                 uint64_t *keys, DevStatus *st, cudaStream_t s)
{
    k_keys<<<(N + 255) / 256, 256, 0, s>>>(pos, N, box_off, nbox, bps, keys, st);
    g_launches++;
}

// ------------------------------------------------------------------ radix sort
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 12;
constexpr int kRsTile = kRsThreads * kRsItems;  // 3072 pairs per block

size_t radix_hist_elems(uint32_t n) { return (size_t)256 * ((n + kRsTile - 1) / kRsTile) + 1; }

// SRC 0: digit = key bits [shift, shift+8); SRC 1: digit = bits of the box of the value.
template <int SRC>
__device__ __forceinline__ uint32_t rs_digit(uint64_t k, uint32_t v, int shift, const uint32_t *box_off, int nbox)
{
    if (SRC == 0) return (uint32_t)(k >> shift) & 255u;
    return ((uint32_t)box_of(v, box_off, nbox) >> shift) & 255u;
}

template <int SRC>
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t *__restrict__ key,
                                                         const uint32_t *__restrict__ val, uint32_t n, int shift,
                                                         uint32_t nblk, uint32_t *__restrict__ hist,
                                                         const uint32_t *__restrict__ box_off, int nbox)
{
    __shared__ uint32_t h[kRsWarps][256];
    for (int d = threadIdx.x; d < kRsWarps * 256; d += kRsThreads) (&h[0][0])[d] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const uint32_t base = blockIdx.x * kRsTile;
#pragma unroll 4
    for (int t = 0; t < kRsItems; t++) {
        uint32_t i = base + t * kRsThreads + threadIdx.x;
        if (i < n) {
            uint32_t v = val ? val[i] : i;
            atomicAdd(&h[w][rs_digit<SRC>(key[i], v, shift, box_off, nbox)], 1u);
        }
    }
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ww++) s += h[ww][threadIdx.x];
    hist[(size_t)threadIdx.x * nblk + blockIdx.x] = s;
}

// Stable scatter.  Warp w of a block ranks the pairs [w*kRsItems*32, (w+1)*kRsItems*32)
// of the tile in input order (rounds of 32 consecutive pairs, lanes in order), the block
// places the tile in shared memory in digit order, and the tile is written out in
// contiguous runs per digit.
template <int SRC>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t *__restrict__ kin,
                                                            const uint32_t *__restrict__ vin,
                                                            uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                            uint32_t n, int shift, uint32_t nblk,
                                                            const uint32_t *__restrict__ off,
                                                            const uint32_t *__restrict__ box_off, int nbox)
{
    __shared__ uint32_t wcnt[kRsWarps][256];
    __shared__ uint32_t dstart[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t wsum[kRsWarps];
    __shared__ uint64_t sk[kRsTile];
    __shared__ uint32_t sv[kRsTile];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int d = tid; d < kRsWarps * 256; d += kRsThreads) (&wcnt[0][0])[d] = 0;
    gbase[tid] = off[(size_t)tid * nblk + blockIdx.x];
    __syncthreads();

    uint64_t k[kRsItems];
    uint32_t v[kRsItems], dg[kRsItems], rk[kRsItems];
    const uint32_t wbase = blockIdx.x * kRsTile + w * (kRsItems * 32);
    const unsigned lt = (1u << lane) - 1u;
    // all of this thread's loads are issued before the ranking, which is serialised
    // through shared memory
#pragma unroll
    for (int t = 0; t < kRsItems; t++) {
        const uint32_t i = wbase + t * 32 + lane;
        k[t] = i < n ? kin[i] : 0ull;
        v[t] = i < n ? (vin ? vin[i] : i) : 0u;
    }
#pragma unroll
    for (int t = 0; t < kRsItems; t++) {
        const bool valid = wbase + t * 32 + lane < n;
        uint32_t d = valid ? rs_digit<SRC>(k[t], v[t], shift, box_off, nbox) : 256u;
        dg[t] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = d < 256u ? wcnt[w][d] : 0u;
        __syncwarp();
        if (d < 256u && (peers & lt) == 0u) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        rk[t] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive offsets of the warps, and the tile total
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ww++) {
        uint32_t c = wcnt[ww][tid];
        wcnt[ww][tid] = tot;
        tot += c;
    }
    // exclusive scan of the 256 digit totals -> tile-local digit starts
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t wb = 0;
    for (int ww = 0; ww < w; ww++) wb += wsum[ww];
    dstart[tid] = wb + x - tot;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kRsItems; t++) {
        if (dg[t] < 256u) {
            uint32_t lp = dstart[dg[t]] + wcnt[w][dg[t]] + rk[t];
            sk[lp] = k[t];
            sv[lp] = v[t];
        }
    }
    __syncthreads();
    const uint32_t tbase = blockIdx.x * kRsTile;
    const uint32_t cnt = min((uint32_t)kRsTile, n - tbase);
    for (uint32_t j = tid; j < cnt; j += kRsThreads) {
        uint64_t kk = sk[j];
        uint32_t vv = sv[j];
        uint32_t d = rs_digit<SRC>(kk, vv, shift, box_off, nbox);
        uint32_t gp = gbase[d] + (j - dstart[d]);
        kout[gp] = kk;
        vout[gp] = vv;
    }
}

void radix_sort(uint64_t *k0, uint64_t *k1, uint32_t *v0, uint32_t *v1, uint32_t n, int key_passes, int box_passes,
                const uint32_t *box_off, int nbox, uint32_t *hist, uint32_t *scan_scratch, uint64_t **k_out,
                uint32_t **v_out, cudaStream_t s)
{
    const uint32_t nblk = (n + kRsTile - 1) / kRsTile;
    uint64_t *ki = k0, *ko = k1;
    uint32_t *vi = nullptr, *vo = v1;  // first pass generates the identity values
    uint32_t *vfree = v0;
    const int passes = key_passes + box_passes;
    for (int p = 0; p < passes; p++) {
        const bool boxp = p >= key_passes;
        const int shift = boxp ? 8 * (p - key_passes) : 8 * p;
        if (boxp) {
            k_rs_hist<1><<<nblk, kRsThreads, 0, s>>>(ki, vi, n, shift, nblk, hist, box_off, nbox);
        } else {
            k_rs_hist<0><<<nblk, kRsThreads, 0, s>>>(ki, vi, n, shift, nblk, hist, box_off, nbox);
        }
        g_launches++;
        scan_u32(hist, hist, (size_t)256 * nblk, scan_scratch, s);
        if (boxp) {
            k_rs_scatter<1><<<nblk, kRsThreads, 0, s>>>(ki, vi, ko, vo, n, shift, nblk, hist, box_off, nbox);
        } else {
            k_rs_scatter<0><<<nblk, kRsThreads, 0, s>>>(ki, vi, ko, vo, n, shift, nblk, hist, box_off, nbox);
        }
        g_launches++;
        // ping-pong
        uint64_t *kt = ki;
        ki = ko;
        ko = kt;
        uint32_t *vt = vi ? vi : vfree;
        vi = vo;
        vo = vt;
    }
    *k_out = ki;
    *v_out = vi;
}

// ------------------------------------------------------------------ gather
__global__ void __launch_bounds__(256) k_gather(const double *__restrict__ pos, const float *__restrict__ mass,
                                                const uint32_t *__restrict__ perm, uint32_t N,
                                                const uint32_t *__restrict__ box_off, int nbox,
                                                const BoxPar *__restrict__ bps, double *__restrict__ xs,
                                                double *__restrict__ ys, double *__restrict__ zs,
                                                float *__restrict__ ms, DevStatus *st)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint32_t j = perm[i];
    double L = bps[box_of(i, box_off, nbox)].L;
    xs[i] = wrap_pos_fast(pos[3 * (size_t)j], L);
    ys[i] = wrap_pos_fast(pos[3 * (size_t)j + 1], L);
    zs[i] = wrap_pos_fast(pos[3 * (size_t)j + 2], L);
    const float m = mass[j];
    ms[i] = m;
    // the FP32 force keeps a pair at distance 0 finite only for |m| < 2^38 (and NaN fails too)
    if (!(fabsf(m) < 274877906944.0f)) atomicOr(&st->flags, ST_NONFINITE);
}

void launch_gather(const double *pos, const float *mass, const uint32_t *perm, uint32_t N, const uint32_t *box_off,
                   int nbox, const BoxPar *bps, double *xs, double *ys, double *zs, float *ms, DevStatus *st,
                   cudaStream_t s)
{
    k_gather<<<(N + 255) / 256, 256, 0, s>>>(pos, mass, perm, N, box_off, nbox, bps, xs, ys, zs, ms, st);
    g_launches++;
}

}  // namespace greem
