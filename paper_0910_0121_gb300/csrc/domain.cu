// The multi-process form of the short-range force (Sec. 2.2 steps 3, 4 and 7; Sec. 2.3.1):
// the finest cells of sampled particles for the domain decomposition, the packing of
// particles by destination domain for their redistribution, and the local essential
// tree (LET) that one process exports to the domain of another.
//
// Domains are boxes of finest cells (units L/2^21), half-open per axis, that tile the
// periodic box.  A particle belongs to the box that holds its finest cell (the cell of
// its Morton key, reading C9), so every process decides membership identically.
//
// LET (Sec. 2.2 step 3): the nodes of the local tree that satisfy the opening criterion
// from the surface of the receiving domain and lie within r_cut of it, and the particles
// of opened leaves that lie within r_cut; a node whose ancestor was accepted or pruned is
// not visited.  The tests are the walker's (readings C1, C2, C4) with the domain box in
// place of the group's cell and particle box: prune a node iff its cell's periodic gap to
// the box exceeds r_cut (exact integer threshold T_prune); accept it iff its level is at
// least l_min and the squared distance from its cell centre to the nearest point of the
// box exceeds the level's threshold A[k].  Every node decides from its own cell and its
// ancestors' decisions, so the export is one flat pass over the nodes, not a walk; items
// come out in node preorder (a leaf's particles in sorted order), as a recursive walk
// would emit them.
#include "cells.cuh"
#include "common.cuh"

namespace greem {

constexpr int kDomThreads = 256;
constexpr int kDomWarps = kDomThreads / 32;

// Finest cells of the particles idx[k] (or k) of pos [npos, 3]; an index outside [0, npos)
// or a non-finite coordinate sets ST_NONFINITE (the call returns INVALID_ARG).
__global__ void __launch_bounds__(kDomThreads) k_cells(const double *__restrict__ pos, uint32_t npos,
                                                      const int64_t *__restrict__ idx, uint32_t n, double L,
                                                      double invL, int pow2_e, int32_t *__restrict__ cells,
                                                      DevStatus *st)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t ii = idx ? idx[k] : (int64_t)k;
    if (ii < 0 || ii >= (int64_t)npos) {
        atomicOr(&st->flags, ST_NONFINITE);
        cells[3 * (size_t)k] = cells[3 * (size_t)k + 1] = cells[3 * (size_t)k + 2] = 0;
        return;
    }
    const size_t i = (size_t)ii;
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
        atomicOr(&st->flags, ST_NONFINITE);
        cells[3 * (size_t)k] = cells[3 * (size_t)k + 1] = cells[3 * (size_t)k + 2] = 0;
        return;
    }
    const uint3 c = cells_of(x, y, z, L, invL, pow2_e);
    cells[3 * (size_t)k] = (int32_t)c.x;
    cells[3 * (size_t)k + 1] = (int32_t)c.y;
    cells[3 * (size_t)k + 2] = (int32_t)c.z;
}

void launch_cells(const double *pos, uint32_t npos, const int64_t *idx, uint32_t n, double L, int pow2_e,
                  int32_t *cells, DevStatus *st, cudaStream_t s)
{
    k_cells<<<(n + kDomThreads - 1) / kDomThreads, kDomThreads, 0, s>>>(pos, npos, idx, n, L, 1.0 / L, pow2_e, cells,
                                                                         st);
    g_launches++;
}

// The domain of each particle (the box holding its finest cell) and, per block of
// kDomThreads particles, the count of each domain: cnt[d * nblk + block].  A particle in
// no box (boxes that do not tile) or with a non-finite coordinate flags ST_NONFINITE and
// is counted in domain 0, so that the scatter stays in bounds.
__global__ void __launch_bounds__(kDomThreads) k_dom_count(const double *__restrict__ pos, uint32_t N, double L,
                                                          double invL, int pow2_e, const int32_t *__restrict__ boxes,
                                                          int ndom, uint32_t *__restrict__ dom,
                                                          uint32_t *__restrict__ cnt, DevStatus *st)
{
    extern __shared__ int32_t dsm[];
    int32_t *sbox = dsm;                                          // [ndom * 6]
    uint32_t *hist = reinterpret_cast<uint32_t *>(dsm + 6 * ndom);  // [ndom]
    for (int t = threadIdx.x; t < 6 * ndom; t += blockDim.x) sbox[t] = boxes[t];
    for (int t = threadIdx.x; t < ndom; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const double x = pos[3 * (size_t)i], y = pos[3 * (size_t)i + 1], z = pos[3 * (size_t)i + 2];
        int d = -1;
        if (isfinite(x) && isfinite(y) && isfinite(z)) {
            const uint3 c = cells_of(x, y, z, L, invL, pow2_e);
            for (int q = 0; q < ndom; q++) {
                const int32_t *b = sbox + 6 * q;
                if ((int32_t)c.x >= b[0] && (int32_t)c.x < b[1] && (int32_t)c.y >= b[2] && (int32_t)c.y < b[3] &&
                    (int32_t)c.z >= b[4] && (int32_t)c.z < b[5]) {
                    d = q;
                    break;
                }
            }
        }
        if (d < 0) {
            atomicOr(&st->flags, ST_NONFINITE);
            d = 0;
        }
        dom[i] = (uint32_t)d;
        atomicAdd(&hist[d], 1u);
    }
    __syncthreads();
    const uint32_t nblk = gridDim.x;
    for (int t = threadIdx.x; t < ndom; t += blockDim.x) cnt[(size_t)t * nblk + blockIdx.x] = hist[t];
}

// Stable scatter by domain: off is the exclusive scan of cnt (domain-major), so domain
// d's particles of block b start at off[d * nblk + b]; within a block, warps go in
// order and lanes rank among equal domains by their position.  Positions are written
// wrapped into [0, L).
__global__ void __launch_bounds__(kDomThreads) k_dom_scatter(const double *__restrict__ pos,
                                                            const float *__restrict__ mass,
                                                            const int64_t *__restrict__ ids, uint32_t N, double L,
                                                            const uint32_t *__restrict__ dom,
                                                            const uint32_t *__restrict__ off, int ndom,
                                                            double *__restrict__ pos_out, float *__restrict__ mass_out,
                                                            int64_t *__restrict__ ids_out)
{
    extern __shared__ uint32_t wcnt[];  // [kDomWarps][ndom]
    const unsigned FULL = 0xffffffffu;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < kDomWarps * ndom; t += blockDim.x) wcnt[t] = 0;
    __syncthreads();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool v = i < N;
    const uint32_t d = v ? dom[i] : 0xffffffffu;
    const unsigned peers = __match_any_sync(FULL, d);
    const uint32_t rank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
    if (v && rank == 0) wcnt[w * ndom + d] = (uint32_t)__popc(peers);
    __syncthreads();
    if (!v) return;
    uint32_t dst = off[(size_t)d * gridDim.x + blockIdx.x] + rank;
    for (int ww = 0; ww < w; ww++) dst += wcnt[ww * ndom + d];
    pos_out[3 * (size_t)dst] = wrap_pos_fast(pos[3 * (size_t)i], L);
    pos_out[3 * (size_t)dst + 1] = wrap_pos_fast(pos[3 * (size_t)i + 1], L);
    pos_out[3 * (size_t)dst + 2] = wrap_pos_fast(pos[3 * (size_t)i + 2], L);
    mass_out[dst] = mass[i];
    ids_out[dst] = ids ? ids[i] : (int64_t)i;
}

size_t dom_count_smem(int ndom) { return (size_t)ndom * 7 * sizeof(int32_t); }
size_t dom_scatter_smem(int ndom) { return (size_t)ndom * kDomWarps * sizeof(uint32_t); }
uint32_t dom_blocks(uint32_t N) { return (N + kDomThreads - 1) / kDomThreads; }

void launch_dom_count(const double *pos, uint32_t N, double L, int pow2_e, const int32_t *boxes, int ndom,
                      uint32_t *dom, uint32_t *cnt, DevStatus *st, cudaStream_t s)
{
    k_dom_count<<<dom_blocks(N), kDomThreads, dom_count_smem(ndom), s>>>(pos, N, L, 1.0 / L, pow2_e, boxes, ndom, dom,
                                                                          cnt, st);
    g_launches++;
}

void launch_dom_scatter(const double *pos, const float *mass, const int64_t *ids, uint32_t N, double L,
                        const uint32_t *dom, const uint32_t *off, int ndom, double *pos_out, float *mass_out,
                        int64_t *ids_out, cudaStream_t s)
{
    k_dom_scatter<<<dom_blocks(N), kDomThreads, dom_scatter_smem(ndom), s>>>(pos, mass, ids, N, L, dom, off, ndom,
                                                                              pos_out, mass_out, ids_out);
    g_launches++;
}

// ------------------------------------------------------------------ LET
__device__ __forceinline__ long long wrap_u(long long d)
{
    if (d >= kHalfPeriod) d -= kPeriod;
    else if (d < -kHalfPeriod) d += kPeriod;
    return d;
}

// Squared periodic gap between a cube (centre c, half side h, units u) and the box.
__device__ __forceinline__ long long let_gap2(const LetBox &b, long long cx, long long cy, long long cz, long long h)
{
    const long long c[3] = {cx, cy, cz};
    long long s = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long d = wrap_u(b.c[a] - c[a]);
        d = d < 0 ? -d : d;
        const long long g = d - h - b.h[a];
        if (g > 0) s += g * g;
    }
    return s;
}

// 0 pruned, 1 accepted, 2 opened: the node against the box (C2 prune first, then C1).
__device__ __forceinline__ uint8_t let_status(const Node &nd, const LetBox &b, const BoxPar &bp)
{
    const int k = nd.lvl & 255u;
    const long long hn = 1ll << (kMaxLevel - k);
    const long long cx = 2ll * nd.ix + hn, cy = 2ll * nd.iy + hn, cz = 2ll * nd.iz + hn;
    if (let_gap2(b, cx, cy, cz, hn) > bp.T_prune) return 0;
    const long long c[3] = {cx, cy, cz};
    long long sd = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long d = wrap_u(b.c[a] - c[a]);
        d = d < 0 ? -d : d;
        const long long e = d - b.h[a];
        if (e > 0) sd += e * e;
    }
    if (k >= bp.lmin && sd > bp.A[k]) return 1;
    return 2;
}

__device__ __forceinline__ bool let_particle_in(unsigned long long pc, const LetBox &b, const BoxPar &bp)
{
    const long long fx = (long long)(pc & 0x1fffffull), fy = (long long)((pc >> 21) & 0x1fffffull),
                    fz = (long long)((pc >> 42) & 0x1fffffull);
    return let_gap2(b, 2 * fx + 1, 2 * fy + 1, 2 * fz + 1, 1) <= bp.T_prune;
}

// Up to kLetChunk receiving boxes are handled by one set of passes: a node's status for
// box j sits in bits 2j..2j+1 of its flag word.
struct LetBoxes {
    LetBox b[kLetChunk];
    int n;
};

__global__ void __launch_bounds__(256) k_let_flags(const Node *__restrict__ nodes, const uint32_t *__restrict__ n_nodes,
                                                   uint32_t ncap, LetBoxes bx, const BoxPar *__restrict__ bps,
                                                   uint32_t *__restrict__ flag)
{
    const uint32_t nn = min(*n_nodes, ncap);
    const BoxPar &bp = bps[0];
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += gridDim.x * blockDim.x) {
        const Node nd = nodes[n];
        uint32_t f = 0;
        for (int j = 0; j < bx.n; j++) f |= (uint32_t)let_status(nd, bx.b[j], bp) << (2 * j);
        flag[n] = f;
    }
}

// Boxes (bit j) whose status in the flag word is "opened" (2).
__device__ __forceinline__ uint32_t opened_boxes(uint32_t f, int nb)
{
    uint32_t m = 0;
    for (int j = 0; j < nb; j++) m |= (((f >> (2 * j)) & 3u) == 2u ? 1u : 0u) << j;
    return m;
}

// Items each node contributes to each box, box-major: cnt[j * (ncap + 1) + n].  A node is
// visited for box j when every ancestor was opened for j; then it contributes 1 if it was
// accepted, its particles within r_cut if it is an opened leaf, 0 otherwise.  Entries at
// n >= n_nodes and the last entry of each box's run are 0, so one scan over the whole array
// gives every item its final place, the boxes packed in order.
__global__ void __launch_bounds__(256) k_let_count(const Node *__restrict__ nodes, const uint32_t *__restrict__ n_nodes,
                                                   uint32_t ncap, const uint32_t *__restrict__ flag,
                                                   const unsigned long long *__restrict__ pcell, LetBoxes bx,
                                                   const BoxPar *__restrict__ bps, uint32_t *__restrict__ cnt)
{
    const uint32_t nn = min(*n_nodes, ncap);
    const BoxPar &bp = bps[0];
    const size_t run = (size_t)ncap + 1;
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n <= ncap; n += gridDim.x * blockDim.x) {
        uint32_t vis = 0;
        Node nd;
        uint32_t f = 0;
        if (n < nn) {
            nd = nodes[n];
            f = flag[n];
            vis = (bx.n >= 32 ? 0xffffffffu : ((1u << bx.n) - 1u));
            for (uint32_t q = nd.parent; q != kNone && vis; q = nodes[q].parent) vis &= opened_boxes(flag[q], bx.n);
        }
        for (int j = 0; j < bx.n; j++) {
            uint32_t c = 0;
            if ((vis >> j) & 1u) {
                const uint32_t s = (f >> (2 * j)) & 3u;
                if (s == 1u) c = 1;
                else if (s == 2u && (nd.lvl & 256u))
                    for (uint32_t i = nd.begin; i < nd.end; i++) c += let_particle_in(pcell[i], bx.b[j], bp) ? 1u : 0u;
            }
            cnt[(size_t)j * run + n] = c;
        }
    }
}

__global__ void __launch_bounds__(256) k_let_fill(const Node *__restrict__ nodes, const uint32_t *__restrict__ n_nodes,
                                                  uint32_t ncap, const uint32_t *__restrict__ flag,
                                                  const uint32_t *__restrict__ off,
                                                  const unsigned long long *__restrict__ pcell, LetBoxes bx,
                                                  const BoxPar *__restrict__ bps, const double *__restrict__ xs,
                                                  const double *__restrict__ ys, const double *__restrict__ zs,
                                                  const float *__restrict__ ms, const Dbl4 *__restrict__ mom64,
                                                  double *__restrict__ pos_out, float *__restrict__ mass_out,
                                                  int64_t *__restrict__ ref_out, unsigned long long base)
{
    const uint32_t nn = min(*n_nodes, ncap);
    const BoxPar &bp = bps[0];
    const size_t run = (size_t)ncap + 1;
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += gridDim.x * blockDim.x) {
        for (int j = 0; j < bx.n; j++) {
            const size_t k = (size_t)j * run + n;
            const uint32_t c = off[k + 1] - off[k];
            if (c == 0) continue;
            unsigned long long o = base + off[k];
            if (((flag[n] >> (2 * j)) & 3u) == 1u) {
                const Dbl4 m = mom64[n];
                pos_out[3 * o] = m.x;
                pos_out[3 * o + 1] = m.y;
                pos_out[3 * o + 2] = m.z;
                mass_out[o] = (float)m.w;
                if (ref_out) ref_out[o] = -1 - (int64_t)n;
                continue;
            }
            const Node nd = nodes[n];
            for (uint32_t i = nd.begin; i < nd.end; i++) {
                if (!let_particle_in(pcell[i], bx.b[j], bp)) continue;
                pos_out[3 * o] = xs[i];
                pos_out[3 * o + 1] = ys[i];
                pos_out[3 * o + 2] = zs[i];
                mass_out[o] = ms[i];
                if (ref_out) ref_out[o] = (int64_t)i;
                o++;
            }
        }
    }
}

// The offsets at the ends of the boxes' runs: ends[j] = off[(j + 1) * (ncap + 1) - 1 + 1].
__global__ void k_let_ends(const uint32_t *__restrict__ off, uint32_t ncap, int nb, uint32_t *__restrict__ ends)
{
    const int j = threadIdx.x;
    if (j <= nb) ends[j] = off[(size_t)j * ((size_t)ncap + 1)];
}

void launch_let_count(const Node *nodes, const uint32_t *n_nodes, uint32_t ncap, const LetBox *b, int nb,
                      const BoxPar *bps, const unsigned long long *pcell, uint32_t *flag, uint32_t *cnt, cudaStream_t s,
                      int nsm)
{
    LetBoxes bx;
    bx.n = nb;
    for (int j = 0; j < nb; j++) bx.b[j] = b[j];
    k_let_flags<<<nsm * 8, 256, 0, s>>>(nodes, n_nodes, ncap, bx, bps, flag);
    k_let_count<<<nsm * 8, 256, 0, s>>>(nodes, n_nodes, ncap, flag, pcell, bx, bps, cnt);
    g_launches += 2;
}

void launch_let_ends(const uint32_t *off, uint32_t ncap, int nb, uint32_t *ends, cudaStream_t s)
{
    k_let_ends<<<1, 32, 0, s>>>(off, ncap, nb, ends);
    g_launches++;
}

void launch_let_fill(const Node *nodes, const uint32_t *n_nodes, uint32_t ncap, const LetBox *b, int nb,
                     const BoxPar *bps, const unsigned long long *pcell, const uint32_t *flag, const uint32_t *off,
                     const double *xs, const double *ys, const double *zs, const float *ms, const Dbl4 *mom64,
                     double *pos_out, float *mass_out, int64_t *ref_out, unsigned long long base, cudaStream_t s,
                     int nsm)
{
    LetBoxes bx;
    bx.n = nb;
    for (int j = 0; j < nb; j++) bx.b[j] = b[j];
    k_let_fill<<<nsm * 8, 256, 0, s>>>(nodes, n_nodes, ncap, flag, off, pcell, bx, bps, xs, ys, zs, ms, mom64,
                                       pos_out, mass_out, ref_out, base);
    g_launches++;
}

}  // namespace greem

// ------------------------------------------------------------------ host-only calls
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "greem.h"

namespace {

constexpr int32_t kCells = 1 << 21;

// Cuts of the half-open range [lo, hi) into np parts with equal numbers of the sorted
// values v (the samples inside the range): cut a lies between the values of ranks
// a n/np - 1 and a n/np, rounded up (so equal values stay on one side); parts with no
// samples to go by are cut evenly.  Monotone, cut[0] = lo, cut[np] = hi.
std::vector<int32_t> equal_count_cuts(std::vector<int32_t> v, int np, int32_t lo, int32_t hi)
{
    std::sort(v.begin(), v.end());
    const int64_t n = (int64_t)v.size();
    std::vector<int32_t> cut(np + 1);
    cut[0] = lo;
    cut[np] = hi;
    for (int a = 1; a < np; a++) {
        int32_t c;
        const int64_t k = (int64_t)a * n / np;
        if (n == 0) c = lo + (int32_t)((int64_t)(hi - lo) * a / np);
        else if (k == 0) c = v[0];
        else c = (int32_t)(((int64_t)v[k - 1] + (int64_t)v[k] + 1) / 2);
        c = std::max(c, cut[a - 1]);
        c = std::min(c, hi);
        cut[a] = c;
    }
    return cut;
}

}  // namespace

extern "C" int64_t greem_sample_count(int64_t n_total, int64_t n_local, int nproc, double rate, double t_local,
                                      double t_sum, double alpha)
{
    if (n_total < 0 || n_local < 0 || n_local > n_total || nproc < 1 || !(rate >= 0) || !std::isfinite(rate))
        return -1;
    // Eq. 4: the share of the measured time; equal shares before any time is measured
    const double f = (t_sum > 0 && t_local >= 0 && std::isfinite(t_sum)) ? t_local / t_sum : 1.0 / nproc;
    double n = std::floor((double)n_total * rate * f + 0.5);  // Eq. 3
    if (alpha >= 0) n = std::max(n, std::floor((double)n_local * rate / (1.0 + alpha)));  // Eq. 5
    n = std::min(n, (double)n_local);
    return n < 0 ? 0 : (int64_t)n;
}

extern "C" int greem_domain_boxes(const int32_t *cells, int64_t n, int px, int py, int pz, int32_t *boxes)
{
    if (n < 0 || (n > 0 && !cells) || !boxes || px < 1 || py < 1 || pz < 1) return GREEM_ERR_INVALID_ARG;
    if ((int64_t)px * py * pz > greem::kMaxDomains) return GREEM_ERR_INVALID_ARG;
    for (int64_t i = 0; i < 3 * n; i++)
        if (cells[i] < 0 || cells[i] >= kCells) return GREEM_ERR_INVALID_ARG;
    std::vector<int32_t> v;
    v.reserve((size_t)n);
    for (int64_t i = 0; i < n; i++) v.push_back(cells[3 * i]);
    const std::vector<int32_t> cx = equal_count_cuts(v, px, 0, kCells);
    for (int a = 0; a < px; a++) {
        v.clear();
        for (int64_t i = 0; i < n; i++)
            if (cells[3 * i] >= cx[a] && cells[3 * i] < cx[a + 1]) v.push_back(cells[3 * i + 1]);
        const std::vector<int32_t> cy = equal_count_cuts(v, py, 0, kCells);
        for (int b = 0; b < py; b++) {
            v.clear();
            for (int64_t i = 0; i < n; i++)
                if (cells[3 * i] >= cx[a] && cells[3 * i] < cx[a + 1] && cells[3 * i + 1] >= cy[b] &&
                    cells[3 * i + 1] < cy[b + 1])
                    v.push_back(cells[3 * i + 2]);
            const std::vector<int32_t> cz = equal_count_cuts(v, pz, 0, kCells);
            for (int c = 0; c < pz; c++) {
                int32_t *o = boxes + 6 * (((size_t)a * py + b) * pz + c);
                o[0] = cx[a];
                o[1] = cx[a + 1];
                o[2] = cy[b];
                o[3] = cy[b + 1];
                o[4] = cz[c];
                o[5] = cz[c + 1];
            }
        }
    }
    return GREEM_OK;
}
