// S1 wrap + 63-bit Morton keys, S2 stable LSD radix sort and the SoA gather.
//
// Key (Sec. 3.2.5 "morton key", 12 bytes with the index): each coordinate is wrapped
// into [0, L) (periodic box), mapped to a 21-bit cell index floor((x/L) 2^21) clamped
// to 2^21-1, and the three indices are bit-interleaved with x as the high bit of each
// 3-bit digit.  Every FP64 step uses explicit round-to-nearest intrinsics so that no
// multiply-add is fused: the key is a pure function of the IEEE inputs.
#include <atomic>

#include "cells.cuh"
#include "common.cuh"

namespace greem {

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
        const uint3 c = cells_general(x, y, z, L, invL);
        cx = c.x;
        cy = c.y;
        cz = c.z;
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
// The sort runs in two phases.  Phase A: a stable LSD radix sort of (key, index) pairs on
// the key's top 36 bits (its cells down to level 12), five 8-bit digits, one kernel per
// digit in the
// single-pass ("onesweep") form of decoupled look-back (Merrill & Garland 2016; Adinets
// & Merrill 2022): one pass over the keys histograms every digit at once, then each
// digit pass reads and writes the pairs once.  A block takes the next tile by ticket,
// ranks its pairs, publishes its per-digit counts, and adds up its predecessors' counts
// per digit by looking back through their published words until it meets a published
// inclusive prefix; the tile is then written out in digit order through shared memory.
// Tickets make every block wait only on blocks that started before it.  Each wait has an
// iteration limit, after which the status records a timeout (the call then fails).
// Phase B: the pairs now form runs of equal top bits (particles that share a level-12
// cell), each in input order; every run is sorted by its low 27 bits in place, stably.
// Most runs hold one particle and cost nothing; runs of up to 16 are insertion-sorted by
// the thread at their head, runs of up to 64 by a warp and longer ones by a block (a
// bitonic sort of (low bits, position
// in the run), so equal keys keep their order), and runs beyond a block's shared memory
// by a slower exact one-warp LSD pass over their low bits.  The result is the stable sort
// by the full 63-bit key, whatever the clustering: phase A leaves equal top bits in input
// order and phase B orders each run by the rest of the key.
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
#ifndef GREEM_RS_ITEMS
#define GREEM_RS_ITEMS 12
#endif
#ifndef GREEM_RS_MINB
#define GREEM_RS_MINB 3
#endif
constexpr int kRsItems = GREEM_RS_ITEMS;
constexpr int kRsTile = kRsThreads * kRsItems;  // pairs per tile
constexpr int kRsMaxPasses = 10;                // key digits + up to 2 box digits
constexpr int kRsLowBits = 27;                  // bits left to phase B: levels 13-21
constexpr int kRsKeyPasses = 5;                 // 8-bit digits over the top 36 bits
constexpr int kShortRun = 16;                   // runs sorted by the thread at their head
constexpr int kRunCap = 8192;                   // runs sorted by a block in shared memory
constexpr int kRunThreads = 256;
constexpr size_t kRunSmem = (size_t)kRunCap * (sizeof(uint64_t) + sizeof(uint32_t));
constexpr int kRsLook = 8;                      // predecessors loaded at once in the look-back
constexpr unsigned long long kRsAgg = 1ull << 62, kRsPrefix = 2ull << 62, kRsValue = (1ull << 62) - 1;
constexpr size_t kRsSmem = (size_t)kRsTile * (sizeof(uint64_t) + sizeof(uint32_t));

static inline uint32_t rs_tiles(uint32_t n) { return (n + kRsTile - 1) / kRsTile; }

// u32 words: [passes][256] digit counts, [passes][256] digit starts, [passes] tickets, then
// phase B's counts of long and middle runs and their work counters
size_t radix_hist_elems(uint32_t) { return (size_t)kRsMaxPasses * 512 + kRsMaxPasses + 4; }
// phase B's lists of runs: (start, end) pairs of kShortRun + 1 .. kWarpRun pairs (sorted
// by a warp), then of more (sorted by a block)
constexpr int kWarpRun = 64;
static inline uint32_t mid_cap(uint32_t n) { return n / (kShortRun + 1) + 64; }
static inline uint32_t runs_cap(uint32_t n) { return n / (kWarpRun + 1) + 64; }
size_t radix_runs_elems(uint32_t n) { return 2 * ((size_t)mid_cap(n) + runs_cap(n)); }
int radix_key_passes() { return kRsKeyPasses; }
// u64 look-back words: [passes][tiles][256]
size_t radix_status_elems(uint32_t n) { return (size_t)kRsMaxPasses * rs_tiles(n) * 256; }

// SRC 0: digit = key bits [shift, shift+8); SRC 1: digit = bits of the box of the value.
template <int SRC>
__device__ __forceinline__ uint32_t rs_digit(uint64_t k, uint32_t v, int shift, const uint32_t *box_off, int nbox)
{
    if (SRC == 0) return (uint32_t)(k >> shift) & 255u;
    return ((uint32_t)box_of(v, box_off, nbox) >> shift) & 255u;
}

// Lanes of the warp whose 8-bit digit equals this lane's (d < 256; lanes with d = 256,
// out of range, match only each other): one ballot per digit bit.
__device__ __forceinline__ unsigned digit_peers(uint32_t d)
{
    unsigned peers = __ballot_sync(0xffffffffu, d >= 256u) ^ (d >= 256u ? 0u : 0xffffffffu);
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bb : ~bb;
    }
    return peers;
}

// All digit histograms in one pass over the unsorted keys (the box digits from the box
// of each input index).  A warp whose lanes share a digit adds it with one shared
// atomic (the usual case for the high digits of spatially ordered input); otherwise
// every lane adds its own.
__global__ void __launch_bounds__(256) k_rs_hist_all(const uint64_t *__restrict__ key, uint32_t n, int key_passes,
                                                     int box_passes, const uint32_t *__restrict__ box_off, int nbox,
                                                     uint32_t *__restrict__ hist, int kshift0)
{
    __shared__ uint32_t h[kRsMaxPasses][256];
    const int passes = key_passes + box_passes;
    for (int d = threadIdx.x; d < passes * 256; d += blockDim.x) (&h[0][0])[d] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const uint32_t i = i0 + (uint32_t)lane;
        const bool ok = i < n;
        const uint64_t k = ok ? key[i] : 0ull;
        const uint32_t b = (ok && box_passes) ? (uint32_t)box_of(i, box_off, nbox) : 0u;
        for (int p = 0; p < passes; p++) {
            const uint32_t d = ok ? (p < key_passes ? (uint32_t)(k >> (kshift0 + 8 * p)) & 255u
                                                    : (b >> (8 * (p - key_passes))) & 255u)
                                  : 256u;
            const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
            if (__all_sync(0xffffffffu, d == d0)) {
                if (lane == 0 && d0 < 256u) atomicAdd(&h[p][d0], 32u);
            } else if (ok) {
                atomicAdd(&h[p][d], 1u);
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < passes * 256; d += blockDim.x)
        if ((&h[0][0])[d]) atomicAdd(&hist[d], (&h[0][0])[d]);
}

// Exclusive scan of each pass's 256 counts into its digit starts (one warp per pass).
__global__ void k_rs_digit_starts(uint32_t *hist, int passes)
{
    const int p = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (p >= passes) return;
    const uint32_t *c = hist + p * 256;
    uint32_t *o = hist + kRsMaxPasses * 256 + p * 256;
    uint32_t carry = 0;
    for (int b = 0; b < 256; b += 32) {
        const uint32_t v = c[b + lane];
        uint32_t x = v;
#pragma unroll
        for (int q = 1; q < 32; q <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, q);
            if (lane >= q) x += y;
        }
        o[b + lane] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <int SRC>
__global__ void __launch_bounds__(kRsThreads, GREEM_RS_MINB) k_rs_onesweep(const uint64_t *__restrict__ kin,
                                                             const uint32_t *__restrict__ vin,
                                                             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                             uint32_t n, int shift, const uint32_t *__restrict__ dstart,
                                                             unsigned long long *status, uint32_t *ticket,
                                                             const uint32_t *__restrict__ box_off, int nbox,
                                                             DevStatus *st)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(rs_smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(rs_smem + (size_t)kRsTile * sizeof(uint64_t));
    __shared__ uint32_t wcnt[kRsWarps][256];
    __shared__ uint32_t lstart[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t wsum[kRsWarps];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int d = tid; d < kRsWarps * 256; d += kRsThreads) (&wcnt[0][0])[d] = 0;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;

    uint64_t k[kRsItems];
    uint32_t v[kRsItems], rk[kRsItems];
    const uint32_t wbase = tile * kRsTile + w * (kRsItems * 32);
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int t = 0; t < kRsItems; t++) {
        const uint32_t i = wbase + t * 32 + lane;
        k[t] = i < n ? kin[i] : 0ull;
        v[t] = i < n ? (vin ? vin[i] : i) : 0u;
    }
    // rank within the warp's run of pairs, in input order
#pragma unroll
    for (int t = 0; t < kRsItems; t++) {
        const bool valid = wbase + t * 32 + lane < n;
        const uint32_t d = valid ? rs_digit<SRC>(k[t], v[t], shift, box_off, nbox) : 256u;
        const unsigned peers = digit_peers(d);
        const uint32_t before = d < 256u ? wcnt[w][d] : 0u;
        __syncwarp();
        if (d < 256u && (peers & lt) == 0u) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        rk[t] = valid ? before + __popc(peers & lt) : 0xffffffffu;
    }
    __syncthreads();
    // thread d: warp-exclusive offsets of digit d and the tile's count of d
    uint32_t tot = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ww++) {
        const uint32_t c = wcnt[ww][tid];
        wcnt[ww][tid] = tot;
        tot += c;
    }
    // publish this tile's count at once, so that later tiles need not wait for it
    unsigned long long *my = status + (size_t)tile * 256 + tid;
    if (tile == 0) st_relaxed_u64(my, kRsPrefix | tot);
    else st_relaxed_u64(my, kRsAgg | tot);
    // tile-local digit starts
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t wb = 0;
    for (int ww = 0; ww < w; ww++) wb += wsum[ww];
    lstart[tid] = wb + x - tot;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kRsItems; t++) {
        if (rk[t] != 0xffffffffu) {
            const uint32_t d = rs_digit<SRC>(k[t], v[t], shift, box_off, nbox);
            const uint32_t lp = lstart[d] + wcnt[w][d] + rk[t];
            sk[lp] = k[t];
            sv[lp] = v[t];
        }
    }
    __syncthreads();
    // the tile sits in shared memory in digit order; look back for the exclusive prefix
    // of each digit over the earlier tiles
    if (tile == 0) {
        gbase[tid] = dstart[tid];
    } else {
        // look back over windows of up to kRsLook predecessors, loaded together: add
        // published counts from the nearest one backwards until a published prefix (done)
        // or a tile that has not published yet (wait for it, then go on from there)
        unsigned long long excl = 0;
        int j = (int)tile - 1;
        bool done = false, timeout = false;
        while (!done && !timeout) {
            unsigned long long sw[kRsLook];
#pragma unroll
            for (int q = 0; q < kRsLook; q++)
                sw[q] = j - q >= 0 ? ld_relaxed_u64(status + (size_t)(j - q) * 256 + tid) : kRsPrefix;
            int q = 0;
            for (; q < kRsLook; q++) {
                if ((sw[q] >> 62) == 0ull) break;  // not published yet
                excl += sw[q] & kRsValue;
                if ((sw[q] >> 62) == 2ull) {
                    done = true;
                    break;
                }
            }
            if (done) break;
            j -= q;
            if (q < kRsLook) {
                // wait for tile j to publish (bounded)
                const unsigned long long *w8 = status + (size_t)j * 256 + tid;
                uint32_t it = 0;
                while ((ld_relaxed_u64(w8) >> 62) == 0ull) {
                    if (++it >= kWaitPolls) {
                        atomicOr(&st->flags, ST_TIMEOUT);
                        timeout = true;
                        break;
                    }
                    __nanosleep(32);
                }
            }
        }
        st_relaxed_u64(my, kRsPrefix | (excl + tot));
        gbase[tid] = dstart[tid] + (uint32_t)excl;
    }
    __syncthreads();
    const uint32_t tbase = tile * kRsTile;
    const uint32_t cnt = min((uint32_t)kRsTile, n - tbase);
    for (uint32_t j = tid; j < cnt; j += kRsThreads) {
        const uint64_t kk = sk[j];
        const uint32_t vv = sv[j];
        const uint32_t d = rs_digit<SRC>(kk, vv, shift, box_off, nbox);
        const uint32_t gp = gbase[d] + (j - lstart[d]);
        kout[gp] = kk;
        vout[gp] = vv;
    }
}

// ------------------------------------------------------------------ phase B
__device__ __forceinline__ uint64_t run_top(uint64_t k) { return k >> kRsLowBits; }

// Lanes of the warp whose 9-bit digit equals this lane's (d < 512; d = 512 matches only
// lanes with d = 512).
__device__ __forceinline__ unsigned digit9_peers(uint32_t d)
{
    unsigned peers = __ballot_sync(0xffffffffu, d >= 512u) ^ (d >= 512u ? 0u : 0xffffffffu);
#pragma unroll
    for (int b = 0; b < 9; b++) {
        const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bb : ~bb;
    }
    return peers;
}

// A short run [i, i + len), sorted (stable insertion sort) in place: its few pairs stay in
// the L1 cache.  A real call, so that the threads that only test for a run head (nearly
// all) keep a small register and stack footprint.
static __device__ __noinline__ void sort_short_run(uint64_t *__restrict__ key, uint32_t *__restrict__ val, uint32_t i,
                                                   uint32_t len)
{
    for (uint32_t q = 1; q < len; q++) {
        const uint64_t x = key[i + q];
        const uint32_t y = val[i + q];
        int r = (int)q - 1;
        while (r >= 0 && key[i + r] > x) {
            key[i + r + 1] = key[i + r];
            val[i + r + 1] = val[i + r];
            r--;
        }
        key[i + r + 1] = x;
        val[i + r + 1] = y;
    }
}

// One thread per pair; the thread at the head of a run of two or more sorts a run of up
// to kShortRun pairs itself and lists a longer one, its end found by binary search (the
// top bits are sorted within a box): up to kWarpRun pairs for k_runs_warp (mid, n_mid),
// more for k_runs_long (runs, n_long).  Other threads only read the top bits of pairs that
// runs permute among themselves, so the concurrent sorts do not disturb them.
__global__ void __launch_bounds__(256) k_runs_short(uint64_t *__restrict__ key, uint32_t *__restrict__ val, uint32_t n,
                                                    const uint32_t *__restrict__ box_off, int nbox,
                                                    uint32_t *__restrict__ runs, uint32_t run_cap,
                                                    uint32_t *__restrict__ n_long, uint32_t *__restrict__ mid,
                                                    uint32_t mid_cap_, uint32_t *__restrict__ n_mid)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t t = run_top(key[i]);
    uint32_t e_box = n;
    bool head = i == 0 || run_top(key[i - 1]) != t;
    if (nbox > 1) {
        const int b = box_of(i, box_off, nbox);
        e_box = box_off[b + 1];
        if (box_off[b] == i) head = true;
    }
    if (!head || i + 1 >= e_box || run_top(key[i + 1]) != t) return;  // not a head, or a run of one
    uint32_t e = i + 2;
    while (e < e_box && e - i <= (uint32_t)kShortRun && run_top(key[e]) == t) e++;
    if (e - i <= (uint32_t)kShortRun) {
        sort_short_run(key, val, i, e - i);
        return;
    }
    uint32_t lo = e, hi = e_box;  // the first index from e on whose top differs (or e_box)
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (run_top(key[mid]) == t) lo = mid + 1;
        else hi = mid;
    }
    if (lo - i <= (uint32_t)kWarpRun) {
        const uint32_t slot = atomicAdd(n_mid, 1u);
        if (slot < mid_cap_) {  // always: each listed run takes more than kShortRun pairs
            mid[2 * slot] = i;
            mid[2 * slot + 1] = lo;
        }
        return;
    }
    const uint32_t slot = atomicAdd(n_long, 1u);
    if (slot < run_cap) {  // always: each listed run takes more than kWarpRun pairs
        runs[2 * slot] = i;
        runs[2 * slot + 1] = lo;
    }
}

// Runs of kShortRun + 1 .. kWarpRun pairs, one warp each: lane l holds the run's pairs l
// and l + 32; a 64-element bitonic network sorts the unique keys (low bits << 14 |
// position), the step between the two halves inside each lane, the others by shuffles;
// then every lane fetches the pairs its sorted keys name.
__global__ void __launch_bounds__(256) k_runs_warp(uint64_t *__restrict__ key, uint32_t *__restrict__ val,
                                                   const uint32_t *__restrict__ mid, uint32_t mid_cap_,
                                                   const uint32_t *__restrict__ n_mid, uint32_t *__restrict__ ctr)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t nm = min(*n_mid, mid_cap_);
    const uint64_t lowmask = (1ull << kRsLowBits) - 1ull;
    for (;;) {
        uint32_t r = 0;
        if (lane == 0) r = atomicAdd(ctr, 1u);
        r = __shfl_sync(FULL, r, 0);
        if (r >= nm) break;
        const uint32_t s = mid[2 * r], len = mid[2 * r + 1] - s;
        const uint32_t e0 = (uint32_t)lane, e1 = (uint32_t)lane + 32u;
        const uint64_t k0 = e0 < len ? key[s + e0] : 0ull, k1 = e1 < len ? key[s + e1] : 0ull;
        const uint32_t v0 = e0 < len ? val[s + e0] : 0u, v1 = e1 < len ? val[s + e1] : 0u;
        const uint64_t top = run_top(__shfl_sync(FULL, k0, 0));
        uint64_t c0 = e0 < len ? ((k0 & lowmask) << 14) | e0 : ~0ull;
        uint64_t c1 = e1 < len ? ((k1 & lowmask) << 14) | e1 : ~0ull;
#pragma unroll
        for (uint32_t kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll
            for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
                if (jj == 32) {  // partners in the same lane; kk = 64: ascending
                    const uint64_t lo_ = c0 < c1 ? c0 : c1, hi_ = c0 < c1 ? c1 : c0;
                    c0 = lo_;
                    c1 = hi_;
                } else {
                    const uint64_t o0 = __shfl_xor_sync(FULL, c0, jj), o1 = __shfl_xor_sync(FULL, c1, jj);
                    const bool lower = (e0 & jj) == 0;  // the same for e1 = e0 + 32
                    const bool up0 = (e0 & kk) == 0, up1 = (e1 & kk) == 0;
                    c0 = (lower == up0) ? (c0 < o0 ? c0 : o0) : (c0 > o0 ? c0 : o0);
                    c1 = (lower == up1) ? (c1 < o1 ? c1 : o1) : (c1 > o1 ? c1 : o1);
                }
            }
        }
        const uint32_t p0 = (uint32_t)(c0 & 0x3fffu), p1 = (uint32_t)(c1 & 0x3fffu);
        const uint64_t a0 = __shfl_sync(FULL, k0, p0 & 31u), b0 = __shfl_sync(FULL, k1, p0 & 31u);
        const uint32_t x0 = __shfl_sync(FULL, v0, p0 & 31u), y0 = __shfl_sync(FULL, v1, p0 & 31u);
        const uint64_t a1 = __shfl_sync(FULL, k0, p1 & 31u), b1 = __shfl_sync(FULL, k1, p1 & 31u);
        const uint32_t x1 = __shfl_sync(FULL, v0, p1 & 31u), y1 = __shfl_sync(FULL, v1, p1 & 31u);
        if (e0 < len) {
            key[s + e0] = (top << kRsLowBits) | ((p0 >> 5) ? (b0 & lowmask) : (a0 & lowmask));
            val[s + e0] = (p0 >> 5) ? y0 : x0;
        }
        if (e1 < len) {
            key[s + e1] = (top << kRsLowBits) | ((p1 >> 5) ? (b1 & lowmask) : (a1 & lowmask));
            val[s + e1] = (p1 >> 5) ? y1 : x1;
        }
    }
}

// The listed runs, one block each: up to kRunCap pairs by a bitonic sort in shared memory
// of (low bits << 14 | position in the run), unique keys whose order is the stable one;
// longer runs by one warp, three stable 9-bit LSD passes over the low 27 bits through the
// other ping-pong buffer (tkey, tval) at the same positions, then copied back.
__global__ void __launch_bounds__(kRunThreads) k_runs_long(uint64_t *__restrict__ key, uint32_t *__restrict__ val,
                                                           uint64_t *__restrict__ tkey, uint32_t *__restrict__ tval,
                                                           const uint32_t *__restrict__ runs, uint32_t run_cap,
                                                           const uint32_t *__restrict__ n_long,
                                                           uint32_t *__restrict__ ctr)
{
    extern __shared__ __align__(16) unsigned char run_smem[];
    uint64_t *comp = reinterpret_cast<uint64_t *>(run_smem);
    uint32_t *vals = reinterpret_cast<uint32_t *>(run_smem + (size_t)kRunCap * sizeof(uint64_t));
    __shared__ uint32_t s_r;
    __shared__ uint64_t s_top;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t nl = min(*n_long, run_cap);
    const uint64_t lowmask = (1ull << kRsLowBits) - 1ull;
    for (;;) {
        if (tid == 0) s_r = atomicAdd(ctr, 1u);
        __syncthreads();
        const uint32_t r = s_r;
        if (r >= nl) break;
        const uint32_t s = runs[2 * r], e = runs[2 * r + 1], len = e - s;
        if (len <= (uint32_t)kRunCap) {
            uint32_t P = 1;
            while (P < len) P <<= 1;
            for (uint32_t j = tid; j < P; j += kRunThreads) {
                if (j < len) {
                    const uint64_t k = key[s + j];
                    comp[j] = ((k & lowmask) << 14) | j;
                    vals[j] = val[s + j];
                } else {
                    comp[j] = ~0ull;
                }
            }
            if (tid == 0) s_top = run_top(key[s]);
            __syncthreads();
            for (uint32_t k2 = 2; k2 <= P; k2 <<= 1) {
                for (uint32_t j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
                    for (uint32_t t = tid; t < P; t += kRunThreads) {
                        const uint32_t u = t ^ j2;
                        if (u > t) {
                            const uint64_t a = comp[t], b = comp[u];
                            const bool asc = (t & k2) == 0;
                            if ((a > b) == asc) {
                                comp[t] = b;
                                comp[u] = a;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (uint32_t j = tid; j < len; j += kRunThreads) {
                const uint64_t c = comp[j];
                key[s + j] = (s_top << kRsLowBits) | (c >> 14);
                val[s + j] = vals[c & 0x3fffu];
            }
        } else if (tid < 32) {
            uint32_t *hist = vals;  // 512 digit starts
            const unsigned lt = (1u << lane) - 1u;
            uint64_t *sk = key, *dk = tkey;
            uint32_t *sv = val, *dv = tval;
            for (int pass = 0; pass < 3; pass++) {
                const int shift = 9 * pass;
                for (int d = lane; d < 512; d += 32) hist[d] = 0;
                __syncwarp();
                for (uint32_t j = s + lane; j < e; j += 32) atomicAdd(&hist[(uint32_t)(sk[j] >> shift) & 511u], 1u);
                __syncwarp();
                uint32_t carry = s;
                for (int b = 0; b < 512; b += 32) {
                    const uint32_t v = hist[b + lane];
                    uint32_t x = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                        if (lane >= o) x += y;
                    }
                    hist[b + lane] = carry + x - v;
                    carry += __shfl_sync(0xffffffffu, x, 31);
                }
                __syncwarp();
                for (uint32_t c0 = s; c0 < e; c0 += 32) {
                    const uint32_t j = c0 + lane;
                    const bool ok = j < e;
                    const uint32_t d = ok ? (uint32_t)(sk[j] >> shift) & 511u : 512u;
                    const unsigned peers = digit9_peers(d);
                    const uint32_t base = ok ? hist[d] : 0u;
                    if (ok) {
                        const uint32_t dst = base + __popc(peers & lt);
                        dk[dst] = sk[j];
                        dv[dst] = sv[j];
                    }
                    __syncwarp();
                    if (ok && (peers & lt) == 0u) hist[d] = base + __popc(peers);
                    __syncwarp();
                }
                uint64_t *tk = sk;
                sk = dk;
                dk = tk;
                uint32_t *tv = sv;
                sv = dv;
                dv = tv;
            }
            // three passes leave the run in tkey/tval
            for (uint32_t j = s + lane; j < e; j += 32) {
                key[j] = tkey[j];
                val[j] = tval[j];
            }
        }
        __syncthreads();
    }
}

void radix_sort(uint64_t *k0, uint64_t *k1, uint32_t *v0, uint32_t *v1, uint32_t n, int key_passes, int box_passes,
                const uint32_t *box_off, int nbox, uint32_t *hist, unsigned long long *status, uint32_t *runs,
                DevStatus *st, uint64_t **k_out, uint32_t **v_out, cudaStream_t s, int nsm)
{
    // the shared-memory opt-in applies to the current device only: set once per device
    static std::atomic<bool> attr_set[kMaxDevices];
    const int dev = current_device_index();
    if (dev < 0 || !attr_set[dev].load()) {
        cudaFuncSetAttribute(k_rs_onesweep<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRsSmem);
        cudaFuncSetAttribute(k_rs_onesweep<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRsSmem);
        cudaFuncSetAttribute(k_runs_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRunSmem);
        if (dev >= 0) attr_set[dev].store(true);
    }
    const uint32_t ntile = rs_tiles(n);
    const int passes = key_passes + box_passes;
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * radix_hist_elems(n), s);
    cudaMemsetAsync(status, 0, sizeof(unsigned long long) * (size_t)passes * ntile * 256, s);
    k_rs_hist_all<<<nsm * 4, 256, 0, s>>>(k0, n, key_passes, box_passes, box_off, nbox, hist, kRsLowBits);
    k_rs_digit_starts<<<1, 32 * passes, 0, s>>>(hist, passes);
    g_launches += 2;
    uint64_t *ki = k0, *ko = k1;
    uint32_t *vi = nullptr, *vo = v1;  // first pass generates the identity values
    uint32_t *vfree = v0;
    for (int p = 0; p < passes; p++) {
        const bool boxp = p >= key_passes;
        const int shift = boxp ? 8 * (p - key_passes) : kRsLowBits + 8 * p;
        const uint32_t *ds = hist + kRsMaxPasses * 256 + p * 256;
        uint32_t *tk = hist + kRsMaxPasses * 512 + p;
        unsigned long long *sw = status + (size_t)p * ntile * 256;
        if (boxp) {
            k_rs_onesweep<1><<<ntile, kRsThreads, kRsSmem, s>>>(ki, vi, ko, vo, n, shift, ds, sw, tk, box_off, nbox, st);
        } else {
            k_rs_onesweep<0><<<ntile, kRsThreads, kRsSmem, s>>>(ki, vi, ko, vo, n, shift, ds, sw, tk, box_off, nbox, st);
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
    // phase B: each run of equal top bits by its low bits, in place in (ki, vi); ko and vo
    // hold nothing that is still needed and serve the one-warp path as scratch
    uint32_t *n_long = hist + kRsMaxPasses * 512 + kRsMaxPasses;  // n_long, long work, n_mid, mid work
    uint32_t *mid = runs + 2 * (size_t)runs_cap(n);
    k_runs_short<<<(n + 255) / 256, 256, 0, s>>>(ki, vi, n, box_off, nbox, runs, runs_cap(n), n_long, mid, mid_cap(n),
                                                  n_long + 2);
    k_runs_warp<<<nsm * 4, 256, 0, s>>>(ki, vi, mid, mid_cap(n), n_long + 2, n_long + 3);
    k_runs_long<<<nsm, kRunThreads, kRunSmem, s>>>(ki, vi, ko, vo, runs, runs_cap(n), n_long, n_long + 1);
    g_launches += 3;
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
