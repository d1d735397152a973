// S5 Barnes (1990) grouped interaction lists (Sec. 2.2 steps 3 and 5; Sec. 3.1.2).
//
// One warp per group walks its box's tree from the root with a per-warp stack.  Every
// node the recursive walk visits is tested, in this order:
//   prune  -- the node's cell is farther than r_cut from the group's particle box (the
//             box of finest-level cells that holds the group's particles; periodic
//             box-to-box distance), so none of its particles can act (Eq. 2 is 0);
//   accept -- level >= l_min and the opening criterion holds: cell side l and the
//             distance d from the node's cell centre to the nearest point of the group
//             cell satisfy l < theta d; the node enters the list as one particle at its
//             centre of mass (Sec. 3.1.2);
//   leaf   -- an opened leaf puts its particles into the list, each but those whose
//             finest cell passes the prune test (the same integer test at level 21);
//   open   -- the node's children are tested next.
// No node inside a pruned or accepted subtree is tested.  The entries are the same set
// as the recursive walk's; their order within a list is the order of the steps (the
// debug dump sorts each list back into preorder, i.e. by first particle).
// Every test is done in integer units u = L/2^22 against thresholds the host derives
// from the FP64 comparisons (double)S*u*u > r_cut*r_cut and (double)l*l < theta*theta*S,
// so the lists are exact and bit-identical to a sequential FP64 walk.
//
// Entries are written as float4 (x, y, z, m) relative to the group's cell centre in
// r_cut units (Sec. 3.1.1: positions passed relative to the group centre): the cell
// offset (an exact integer in u, wrapped to the nearest image) times u/r_cut, plus the
// particle's FP32 offset from its own leaf centre (or the node's COM offset from its
// cell centre).  The group's own particles get the same float4 in irel[], so a
// particle and its own list entry are bit-identical and the self pair has r = 0.
//
// Lists are contiguous per group inside pages handed out by an atomic counter; a list
// that does not fit the warp's current page is walked again into fresh pages.
//
// The walk may start below the root.  Let K be a level at or above the first level at
// which any node can be accepted: with the group's particle box inside its cell, a node of
// half side h that passes the prune test lies at squared distance at most
// (sqrt(T_prune) + sqrt(3) h)^2 from the group cell, so no node of a level k with that
// bound <= A[k] (or k < l_min) is ever accepted, and every node above level K that the
// recursive walk reaches is opened or, for a leaf, emptied.  A node below the root that
// passes the prune test has every ancestor passing it too, as long as no ancestor's nearest
// image differs from the image that holds the node; for an ancestor of half side <= L/4
// that holds when L/4 > sqrt(T_prune) + the particle box's half side + its offset from
// the cell centre, on every axis.  Under those two conditions the walk's entries are the
// level-K nodes that pass their tests (and the leaves above level K that pass the prune
// test) taken as the first step, which k_start_table makes a lookup: the level-K cells
// within r_cut of the group's particle box are enumerated, each names its node (or the
// leaf above it, taken once), and the children of the root down to level K are never
// tested.  A group that fails a condition, or whose cells are too many, walks from the
// root.
#include <algorithm>

#include "common.cuh"

namespace greem {

__device__ __forceinline__ int wrap_delta(int d, int &sh)
{
    sh = 0;
    if (d >= kHalfPeriod) {
        d -= kPeriod;
        sh = -1;
    } else if (d < -kHalfPeriod) {
        d += kPeriod;
        sh = 1;
    }
    return d;
}

__device__ __forceinline__ unsigned shift_code(int sx, int sy, int sz)
{
    auto c = [](int s) -> unsigned { return s == 0 ? 0u : (s > 0 ? 1u : 2u); };
    return c(sx) | (c(sy) << 2) | (c(sz) << 4);
}

__device__ __forceinline__ Node load_node(const Node *p)
{
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
    uint4 a = __ldg(q), b = __ldg(q + 1);
    Node n;
    n.ix = a.x; n.iy = a.y; n.iz = a.z; n.lvl = a.w;
    n.begin = b.x; n.end = b.y; n.skip = b.z; n.parent = b.w;
    return n;
}

// Geometry of a cell against the group: the offset of its centre from the group's cell
// centre (u, wrapped to the nearest image; with SHIFT also the image's shift code, which
// only index entries record), the squared gap to the group's particle box, and the
// squared distance from its centre to the group cell (both in u^2).  cell_gap computes
// what the prune test needs; the accept distance follows only for cells that pass it.
struct CellTest {
    int dx, dy, dz;
    unsigned shc;
    long long Sg;
};

// rx, ry, rz: the cell centre minus the group's cell centre (u), before wrapping; h: the
// cell's half side (u).
template <bool SHIFT>
__device__ __forceinline__ CellTest cell_gap(int rx, int ry, int rz, int h, const Group &gr, const int4 tb,
                                             const int4 th)
{
    CellTest c;
    int sx, sy, sz;
    c.dx = wrap_delta(rx, sx);
    c.dy = wrap_delta(ry, sy);
    c.dz = wrap_delta(rz, sz);
    c.shc = SHIFT ? shift_code(sx, sy, sz) : 0u;
    const int gx = max(0, abs(c.dx - tb.x) - h - th.x), gy = max(0, abs(c.dy - tb.y) - h - th.y),
              gz = max(0, abs(c.dz - tb.z) - h - th.z);
    c.Sg = (long long)gx * gx + (long long)gy * gy + (long long)gz * gz;
    return c;
}

__device__ __forceinline__ long long cell_dist2(const CellTest &c, const Group &gr)
{
    const int ex = max(0, abs(c.dx) - gr.hg), ey = max(0, abs(c.dy) - gr.hg), ez = max(0, abs(c.dz) - gr.hg);
    return (long long)ex * ex + (long long)ey * ey + (long long)ez * ez;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// The lane s whose exclusive offset off is the largest one <= t (offsets non-decreasing).
__device__ __forceinline__ int owner_lane(uint32_t off, uint32_t t)
{
    int s = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const uint32_t oc = __shfl_sync(0xffffffffu, off, s + step);
        if (oc <= t) s += step;
    }
    return s;
}

// ---------------------------------------------------------------- start tables
constexpr uint32_t kCoarseLeaf = 0x80000000u;  // table entry: a leaf above level K
constexpr uint32_t kMaxStartCells = 512;       // more candidate cells: walk from the root

// A list warp's counters, kept in shared memory by its lane 0 and added to the status
// word once, when the warp runs out of groups.
enum { kTallyPadded, kTallyLen, kTallyInter, kTallyStart, kTallyN };

// A 10-bit integer's bits spread to every third bit (Morton interleave).
__device__ __forceinline__ uint32_t spread_bits3(uint32_t v)
{
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t cell_morton(uint32_t x, uint32_t y, uint32_t z)
{
    return (spread_bits3(x) << 2) | (spread_bits3(y) << 1) | spread_bits3(z);
}

// One thread per level-(K-1) cell of a box: the descent from the root to the node of
// that cell gives the entries of its 8 level-K children, written as two 16-byte stores.
__global__ void __launch_bounds__(256) k_start_table(const Node *__restrict__ nodes, const uint32_t *__restrict__ kids,
                                                     const uint32_t *__restrict__ base,
                                                     const BoxPar *__restrict__ bps, int nbox,
                                                     uint32_t *__restrict__ tbl, const DevStatus *__restrict__ st)
{
    if (st->flags & ST_NODE_CAP) return;  // the tree is incomplete; the lists are not walked
    for (int b = blockIdx.y; b < nbox; b += gridDim.y) {
        const BoxPar &bp = bps[b];
        const int K = bp.kstart;
        if (K < 2) continue;
        const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
        if (c >= (1u << (3 * (K - 1)))) continue;
        uint32_t r = base[bp.p_begin];  // the box's root
        bool empty = false;
        for (int d = 1; d < K; d++) {
            const uint32_t lv = nodes[r].lvl;
            if (lv & 256u) break;  // a leaf above level K-1 holds the cell
            const uint32_t oct = (c >> (3 * (K - 1 - d))) & 7u;
            const uint32_t mask = (lv >> 16) & 255u;
            if (!(mask & (1u << oct))) {
                empty = true;
                break;
            }
            r = kids[(size_t)r * 8 + __popc(mask & ((1u << oct) - 1u))];
        }
        uint32_t e[8];
        const uint32_t lv = nodes[r].lvl;
#pragma unroll
        for (int o = 0; o < 8; o++) {
            if (empty) e[o] = kNone;
            else if (lv & 256u) e[o] = r | kCoarseLeaf;
            else {
                const uint32_t mask = (lv >> 16) & 255u;
                e[o] = (mask & (1u << o)) ? kids[(size_t)r * 8 + __popc(mask & ((1u << o) - 1u))] : kNone;
            }
        }
        uint4 *dst = reinterpret_cast<uint4 *>(tbl + bp.tbl_off + (size_t)c * 8);
        dst[0] = make_uint4(e[0], e[1], e[2], e[3]);
        dst[1] = make_uint4(e[4], e[5], e[6], e[7]);
    }
}

void launch_start_table(const Node *nodes, const uint32_t *kids, const uint32_t *base, const BoxPar *bps, int nbox,
                        int kmax, uint32_t *tbl, const DevStatus *st, cudaStream_t s)
{
    if (kmax < 2 || nbox < 1) return;
    const uint32_t cells = 1u << (3 * (kmax - 1));
    const dim3 grid((cells + 255) / 256, (unsigned)std::min(nbox, 65535));
    k_start_table<<<grid, 256, 0, s>>>(nodes, kids, base, bps, nbox, tbl, st);
    g_launches++;
}

// One tested cell per lane: an accepted node becomes one entry at its centre of mass
// (acc), a node to open or a leaf to empty goes onto the stack (push).  Returns false
// when the stack would overflow (the status is set; the call is retried).
template <bool INDEX>
__device__ __forceinline__ bool take_cells(const ListArgs &a, bool acc, bool push, uint32_t child, const CellTest &ct,
                                           float kf, unsigned long long pos0, unsigned long long lim, unsigned lt,
                                           uint32_t &cnt, uint32_t &nacc, uint32_t *__restrict__ stk, uint32_t &sp,
                                           uint32_t cap)
{
    const unsigned FULL = 0xffffffffu;
    const unsigned ab = __ballot_sync(FULL, acc);
    if (acc) {
        const unsigned long long p = pos0 + cnt + __popc(ab & lt);
        const float4 v = __ldg(a.noff + child);
        const float4 e = make_float4(__fadd_rn(__fmul_rn((float)ct.dx, kf), v.x),
                                     __fadd_rn(__fmul_rn((float)ct.dy, kf), v.y),
                                     __fadd_rn(__fmul_rn((float)ct.dz, kf), v.z), v.w);
        if (p < lim) {
            a.flist[p] = e;
            if (INDEX) a.ilist[p] = (unsigned long long)child | (1ull << 32) | ((unsigned long long)ct.shc << 33);
        }
    }
    cnt += __popc(ab);
    nacc += __popc(ab);
    const unsigned pb = __ballot_sync(FULL, push);
    if (sp + __popc(pb) > cap) {
        if (lt == 0u) atomicOr(&a.st->flags, ST_STACK);
        return false;
    }
    if (push) stk[sp + __popc(pb & lt)] = child;
    sp += __popc(pb);
    return true;
}

// The first step of a walk that starts at level K = bp.kstart (see the header): the
// level-K cells within r_cut of the group's particle box, tested like the children of an
// opened node.  Returns false if the group must walk from the root instead (sp is then
// untouched); sets overflow on a stack overflow.
template <bool INDEX>
__device__ __forceinline__ bool start_cells(const ListArgs &a, const Group &gr, const int4 tb, const int4 th,
                                            const BoxPar &bp, uint32_t *__restrict__ stk, unsigned long long pos0,
                                            unsigned long long lim, int lane, unsigned lt, uint32_t &cnt,
                                            uint32_t &nacc, uint32_t &sp, bool &overflow)
{
    const int K = bp.kstart;
    if (K < 2) return false;
    const int R = bp.rprune;
    const int quarter = kPeriod / 4;
    if (quarter - th.x - abs(tb.x) <= R || quarter - th.y - abs(tb.y) <= R || quarter - th.z - abs(tb.z) <= R)
        return false;
    const int sh = 22 - K, nK = 1 << K;
    const uint32_t mK = (uint32_t)nK - 1u;
    // per axis: the level-K cells whose gap to the particle box is at most R (unwrapped
    // indices from c0, n of them; the whole axis once if that many reach around)
    auto range = [&](int gc, int t0, int t1, int &c0, int &n) {
        const int lo = gc + t0 - t1 - R, hi = gc + t0 + t1 + R;
        c0 = (lo - 1) >> sh;
        n = (hi >> sh) - c0 + 1;
        if (n >= nK) {
            c0 = 0;
            n = nK;
        }
    };
    int cx0, nx, cy0, ny, cz0, nz;
    range(gr.cx, tb.x, th.x, cx0, nx);
    range(gr.cy, tb.y, th.y, cy0, ny);
    range(gr.cz, tb.z, th.z, cz0, nz);
    const uint32_t ncand = (uint32_t)(nx * ny * nz);
    if (ncand > kMaxStartCells) return false;
    const uint32_t *tb_k = a.tbl + bp.tbl_off;
    const long long Tp = bp.T_prune;
    const int hK = 1 << (kMaxLevel - K);  // half side of a level-K cell (u)
    const bool acc_level = K >= bp.lmin;
    const long long AK = bp.A[K];
    const float kf = bp.k_f;
    // lane's candidate t = (ix ny + iy) nz + iz, advanced by 32 per chunk
    int iz = lane % nz, iy = (lane / nz) % ny, ix = lane / (nz * ny);
    const int sz = 32 % nz, qz = 32 / nz, sy = qz % ny, sx = qz / ny;
    for (uint32_t c0 = 0; c0 < ncand; c0 += 32) {
        const uint32_t t = c0 + (uint32_t)lane;
        bool acc = false, push = false, node_coarse = false;
        uint32_t node = 0;
        CellTest ct;
        ct.dx = ct.dy = ct.dz = 0;
        ct.shc = 0;
        if (t < ncand) {
            const uint32_t wx = (uint32_t)(cx0 + ix) & mK, wy = (uint32_t)(cy0 + iy) & mK,
                           wz = (uint32_t)(cz0 + iz) & mK;
            const uint32_t e = __ldg(tb_k + cell_morton(wx, wy, wz));
            if (e != kNone) {
                if (e & kCoarseLeaf) {
                    // a leaf above level K: tested once, from the first of its cells among
                    // the candidates (per axis, the first index whose cell is in its block)
                    node = e & ~kCoarseLeaf;
                    node_coarse = true;
                    const Node nd = load_node(a.nodes + node);
                    const int kl = (int)(nd.lvl & 255u);
                    const uint32_t bs = 1u << (K - kl);
                    auto first = [&](uint32_t a0, int c0a) -> int {
                        const uint32_t w = (uint32_t)c0a & mK;
                        return ((w - a0) & mK) < bs ? 0 : (int)((a0 - w) & mK);
                    };
                    const int fsh = kMaxLevel - K;
                    if (ix == first(nd.ix >> fsh, cx0) && iy == first(nd.iy >> fsh, cy0) &&
                        iz == first(nd.iz >> fsh, cz0)) {
                        const int hl = 1 << (kMaxLevel - kl);
                        ct = cell_gap<INDEX>(2 * (int)nd.ix + hl - gr.cx, 2 * (int)nd.iy + hl - gr.cy,
                                             2 * (int)nd.iz + hl - gr.cz, hl, gr, tb, th);
                        push = ct.Sg <= Tp;
                    }
                } else {
                    node = e;
                    ct = cell_gap<INDEX>((int)(wx << sh) + hK - gr.cx, (int)(wy << sh) + hK - gr.cy,
                                         (int)(wz << sh) + hK - gr.cz, hK, gr, tb, th);
                    if (ct.Sg <= Tp) {
                        acc = acc_level && cell_dist2(ct, gr) > AK;
                        push = !acc;
                    }
                }
            }
        }
        if (!take_cells<INDEX>(a, acc, push, node, ct, kf, pos0, lim, lt, cnt, nacc, stk, sp, a.stack_cap)) {
            overflow = true;
            break;
        }
        if (INDEX) {
            // a count for tests (each walk of a group counts: the rare walk into fresh
            // pages counts twice)
            const unsigned cb = __ballot_sync(0xffffffffu, push && node_coarse);
            if (cb && lt == 0u) atomicAdd(&a.st->sum_coarse, (unsigned long long)__popc(cb));
        }
        iz += sz;
        const int cz = iz >= nz;
        iz -= cz ? nz : 0;
        iy += sy + cz;
        const int cy = iy >= ny;
        iy -= cy ? ny : 0;
        ix += sx + cy;
    }
    return true;
}

// Walks one group's list; writes entries [pos0, pos0+total) clipped at lim; returns
// total.  stk is this warp's stack (a.stack_cap entries); an overflow sets the status.
//
// The stack holds nodes that passed the prune test and failed the accept test: leaves,
// whose particles are emitted, and nodes to open.  Each step pops up to 32 of them, one
// per lane.  The children of the opened nodes are then spread over the lanes, 32 at a
// time: a child's cell follows from its parent's cell and its octant (the parent's
// child-octant mask), so prune and accept are decided without loading the child; an
// accepted child is written as one entry at its centre of mass, and the others are
// pushed.  Last, the particles of the popped leaves are spread over the lanes and each
// goes through the per-particle r_cut test unless its whole leaf lies within r_cut.
// INDEX: the index entries are written too (a.ilist).
template <bool INDEX>
__device__ uint32_t walk_group(const ListArgs &a, const Group &gr, const int4 tb, const int4 th, const BoxPar &bp,
                               uint32_t root, uint32_t *__restrict__ stk, const uint8_t *__restrict__ octq,
                               unsigned long long pos0, unsigned long long lim, int lane, uint32_t &nacc,
                               bool &from_table)
{
    const unsigned FULL = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    nacc = 0;
    const uint32_t gend = gr.begin + gr.count;
    const long long Tp = bp.T_prune;
    const int lmin = bp.lmin;
    const float kf = bp.k_f;
    const uint32_t cap = a.stack_cap;
    uint32_t cnt = 0;
    uint32_t sp = 0;
    bool overflow = false;
    from_table = start_cells<INDEX>(a, gr, tb, th, bp, stk, pos0, lim, lane, lt, cnt, nacc, sp, overflow);
    if (!from_table) {
        if (lane == 0) stk[0] = root;
        sp = 1;
    }
    __syncwarp();
    while (sp > 0 && !overflow) {
        const uint32_t nb = min(sp, 32u);
        const uint32_t sbase = sp - nb;
        const bool valid = (uint32_t)lane < nb;
        const uint32_t m = valid ? stk[sbase + lane] : 0u;
        __syncwarp();
        sp = sbase;
        Node nd;
        if (valid) {
            nd = load_node(a.nodes + m);
        } else {
            nd.ix = nd.iy = nd.iz = 0; nd.lvl = 0; nd.begin = nd.end = nd.skip = 0; nd.parent = 0;
        }
        const int k = nd.lvl & 255u;
        const bool leaf = valid && (nd.lvl & 256u) != 0;
        const uint32_t mask = valid && !leaf ? (nd.lvl >> 16) & 255u : 0u;
        // the popped node's centre minus the group's cell centre (u, before wrapping)
        const int hn = 1 << (kMaxLevel - k);
        const int ncx = 2 * (int)nd.ix + hn - gr.cx, ncy = 2 * (int)nd.iy + hn - gr.cy, ncz = 2 * (int)nd.iz + hn - gr.cz;

        // ---- children of the opened nodes: prune, accept (one entry), or push
        const uint32_t nch = __popc(mask);
        const uint32_t csum = warp_incl_scan(nch, lane);
        const uint32_t coff = csum - nch;
        const uint32_t ctot = __shfl_sync(FULL, csum, 31);
        for (uint32_t c0 = 0; c0 < ctot; c0 += 32) {
            const uint32_t t = c0 + lane;
            const int s = owner_lane(coff, t);
            const uint32_t o_s = __shfl_sync(FULL, coff, s);
            const int pcx = __shfl_sync(FULL, ncx, s), pcy = __shfl_sync(FULL, ncy, s),
                      pcz = __shfl_sync(FULL, ncz, s);
            const uint32_t plvl = __shfl_sync(FULL, nd.lvl, s), pm = __shfl_sync(FULL, m, s);
            bool acc = false, push = false;
            uint32_t child = 0;
            CellTest ct;
            if (t < ctot) {
                const uint32_t q = t - o_s;
                const uint32_t oct = octq[((plvl >> 13) & (255u << 3)) | q];
                const int kc = (int)(plvl & 255u) + 1;
                const int hc = 1 << (kMaxLevel - kc);
                // a child's centre is its parent's shifted by +-hc per axis
                ct = cell_gap<INDEX>(pcx + ((oct & 4u) ? hc : -hc), pcy + ((oct & 2u) ? hc : -hc),
                                     pcz + ((oct & 1u) ? hc : -hc), hc, gr, tb, th);
                if (ct.Sg <= Tp) {
                    child = __ldg(a.kids + (size_t)pm * 8 + q);
                    acc = kc >= lmin && cell_dist2(ct, gr) > bp.A[kc];
                    push = !acc;
                }
            }
            if (!take_cells<INDEX>(a, acc, push, child, ct, kf, pos0, lim, lt, cnt, nacc, stk, sp, cap)) {
                overflow = true;  // the caller's list is incomplete; the call is retried with a larger stack
                break;
            }
        }
        __syncwarp();
        if (overflow) break;

        // ---- particles of the popped leaves
        uint32_t ne = 0;
        float bx = 0.f, by = 0.f, bz = 0.f;
        unsigned shc = 0;   // test flag in bit 6; INDEX: the leaf's shift code in bits 0-5
        int ox = 0, oy = 0, oz = 0;
        if (leaf) {
            const int h = hn;
            const CellTest lc = cell_gap<INDEX>(ncx, ncy, ncz, h, gr, tb, th);
            // the box of the leaf's particles (finest cells, in slots of q; k_leaf_boxes),
            // its centre relative to the group's cell centre in the leaf's image and its
            // half sides (u): beyond r_cut of the group's particle box, no particle is
            // kept; within it, every particle is (each particle's finest cell is inside)
            const unsigned long long lb = __ldg(a.lbox + m);
            const int q = h > 256 ? (h >> 8) : 1;
            const int lx = (int)(lb & 255u), ly = (int)((lb >> 16) & 255u), lz = (int)((lb >> 32) & 255u);
            const int ux = (int)((lb >> 8) & 255u), uy = (int)((lb >> 24) & 255u), uz = (int)((lb >> 40) & 255u);
            const int bcx = lc.dx - h + (lx + ux + 1) * q - tb.x, bcy = lc.dy - h + (ly + uy + 1) * q - tb.y,
                      bcz = lc.dz - h + (lz + uz + 1) * q - tb.z;
            const int bhx = (ux + 1 - lx) * q, bhy = (uy + 1 - ly) * q, bhz = (uz + 1 - lz) * q;
            const int gx = max(0, abs(bcx) - bhx - th.x), gy = max(0, abs(bcy) - bhy - th.y),
                      gz = max(0, abs(bcz) - bhz - th.z);
            const bool none = (long long)gx * gx + (long long)gy * gy + (long long)gz * gz > Tp;
            const int fx = max(0, abs(bcx) + bhx - th.x), fy = max(0, abs(bcy) + bhy - th.y),
                      fz = max(0, abs(bcz) + bhz - th.z);
            const bool test_each = (long long)fx * fx + (long long)fy * fy + (long long)fz * fz > Tp;
            ne = none ? 0u : nd.end - nd.begin;
            bx = __fmul_rn((float)lc.dx, kf);
            by = __fmul_rn((float)lc.dy, kf);
            bz = __fmul_rn((float)lc.dz, kf);
            shc = lc.shc | (test_each ? 64u : 0u);
            // a particle in finest cell c of this leaf sits at 2c + o (u) from the centre of
            // the group's particle box, in the leaf's image
            ox = lc.dx - ncx - gr.cx + 1 - tb.x;
            oy = lc.dy - ncy - gr.cy + 1 - tb.y;
            oz = lc.dz - ncz - gr.cz + 1 - tb.z;
        }
        const uint32_t isum = warp_incl_scan(ne, lane);
        const uint32_t off = isum - ne;
        const uint32_t tot = __shfl_sync(FULL, isum, 31);
        for (uint32_t t0 = 0; t0 < tot; t0 += 32) {
            const uint32_t t = t0 + lane;
            const int s = owner_lane(off, t);
            const uint32_t o_s = __shfl_sync(FULL, off, s);
            const uint32_t b_s = __shfl_sync(FULL, nd.begin, s);
            const float bx_s = __shfl_sync(FULL, bx, s), by_s = __shfl_sync(FULL, by, s),
                        bz_s = __shfl_sync(FULL, bz, s);
            const unsigned sh_s = __shfl_sync(FULL, shc, s);
            const int ox_s = __shfl_sync(FULL, ox, s), oy_s = __shfl_sync(FULL, oy, s), oz_s = __shfl_sync(FULL, oz, s);
            bool keep = false;
            float4 e;
            uint32_t j = kNone;
            if (t < tot) {
                j = b_s + (t - o_s);
                const float4 v = __ldg(a.poff + j);
                keep = true;
                if (sh_s & 64u) {
                    // the particle's finest cell, in its leaf's image, against the particle box
                    const unsigned long long c = __ldg(a.pcell + j);
                    const int px = 2 * (int)((uint32_t)c & 0x1fffffu) + ox_s;
                    const int py = 2 * (int)((uint32_t)(c >> 21) & 0x1fffffu) + oy_s;
                    const int pz = 2 * (int)(uint32_t)(c >> 42) + oz_s;
                    const int qx = max(0, abs(px) - 1 - th.x), qy = max(0, abs(py) - 1 - th.y),
                              qz = max(0, abs(pz) - 1 - th.z);
                    keep = (long long)qx * qx + (long long)qy * qy + (long long)qz * qz <= Tp;
                }
                e = make_float4(__fadd_rn(bx_s, v.x), __fadd_rn(by_s, v.y), __fadd_rn(bz_s, v.z), v.w);
                if (j >= gr.begin && j < gend) a.irel[j] = e;
            }
            const unsigned kb = __ballot_sync(FULL, keep);
            if (keep) {
                const unsigned long long p = pos0 + cnt + __popc(kb & lt);
                if (p < lim) {
                    a.flist[p] = e;
                    if (INDEX) a.ilist[p] = (unsigned long long)j | ((unsigned long long)(sh_s & 63u) << 33);
                }
            }
            cnt += __popc(kb);
        }
    }
    __syncwarp();
    return cnt;
}

template <bool INDEX>
__global__ void __launch_bounds__(kListWarps * 32, kListBlocksPerSM) k_lists(ListArgs a)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // octq[8 mask + q]: the octant of the (q+1)-th set bit of an 8-bit child mask
    __shared__ uint8_t octq[256 * 8];
    for (uint32_t m = threadIdx.x; m < 256; m += blockDim.x) {
        uint32_t q = 0;
        for (uint32_t o = 0; o < 8; o++)
            if (m & (1u << o)) octq[8 * m + q++] = (uint8_t)o;
        for (; q < 8; q++) octq[8 * m + q] = 0;
    }
    __shared__ unsigned long long tallies[kListWarps][kTallyN];
    if (lane == 0)
        for (int k = 0; k < kTallyN; k++) tallies[threadIdx.x >> 5][k] = 0;
    __syncthreads();
    if (a.st->flags & ST_NODE_CAP) return;  // the tree was truncated: the call is retried
    unsigned long long *tally = tallies[threadIdx.x >> 5];
    const uint32_t G = *a.n_groups;
    uint32_t *stk = a.stack + (size_t)(blockIdx.x * kListWarps + (threadIdx.x >> 5)) * a.stack_cap;
    unsigned long long page_cur = 0, page_end = 0;
    bool exhausted = false;  // the pool ran out: only count what the lists need
    for (;;) {
        unsigned long long gi = 0;
        if (lane == 0) gi = atomicAdd(&a.st->work[0], 1ull);
        gi = __shfl_sync(FULL, gi, 0);
        if (gi >= G) break;
        const uint32_t g = (uint32_t)gi;
        const Group gr = a.groups[g];
        const int4 tb = a.gbox[2 * (size_t)g], th = a.gbox[2 * (size_t)g + 1];
        const BoxPar &bp = a.bps[gr.box];
        const uint32_t root = a.base[bp.p_begin];
        uint32_t nacc = 0;
        bool from_table = false;
        const uint32_t len =
            walk_group<INDEX>(a, gr, tb, th, bp, root, stk, octq, page_cur, page_end, lane, nacc, from_table);
        if (lane == 0) tally[kTallyStart] += from_table ? 1u : 0u;
        const uint32_t padded = (len + 7u) & ~7u;
        if (lane == 0) tally[kTallyPadded] += padded;
        if (exhausted) {
            if (lane == 0) {
                a.loff[g] = 0;
                a.llen[g] = 0;
                a.lraw[g] = 0;
            }
            continue;
        }
        if (page_cur + padded > page_end) {
            unsigned long long np = (padded + a.page - 1) / a.page;
            if (np == 0) np = 1;
            unsigned long long first = 0;
            if (lane == 0) first = atomicAdd(&a.st->list_pages, np);
            first = __shfl_sync(FULL, first, 0);
            if ((first + np) * a.page > a.cap) {
                if (lane == 0) {
                    atomicOr(&a.st->flags, ST_LIST_CAP);
                    a.loff[g] = 0;
                    a.llen[g] = 0;
                    a.lraw[g] = 0;
                }
                page_cur = page_end = 0;
                exhausted = true;
                continue;
            }
            page_cur = first * a.page;
            page_end = (first + np) * a.page;
            walk_group<INDEX>(a, gr, tb, th, bp, root, stk, octq, page_cur, page_end, lane, nacc, from_table);
        }
        for (uint32_t t = len + lane; t < padded; t += 32) {
            a.flist[page_cur + t] = make_float4(16.f, 16.f, 16.f, 0.f);
            if (INDEX) a.ilist[page_cur + t] = ~0ull;
        }
        if (lane == 0) {
            a.loff[g] = page_cur;
            a.llen[g] = padded;
            a.lraw[g] = len;
            if (a.qcnt) a.qcnt[g] = nacc;
            tally[kTallyLen] += len;
            tally[kTallyInter] += (unsigned long long)len * gr.count;
        }
        page_cur += padded;
    }
    __syncwarp();
    if (lane == 0) {
        DevStatus *st = a.st;
        if (tally[kTallyPadded]) atomicAdd(&st->sum_padded, tally[kTallyPadded]);
        if (tally[kTallyLen]) atomicAdd(&st->sum_len, tally[kTallyLen]);
        if (tally[kTallyInter]) atomicAdd(&st->sum_inter, tally[kTallyInter]);
        if (tally[kTallyStart]) atomicAdd(&st->sum_start, tally[kTallyStart]);
    }
}

void launch_lists(const ListArgs &a, cudaStream_t s, int nsm)
{
    if (a.ilist) k_lists<true><<<nsm * kListBlocksPerSM, kListWarps * 32, 0, s>>>(a);
    else k_lists<false><<<nsm * kListBlocksPerSM, kListWarps * 32, 0, s>>>(a);
    g_launches++;
}

}  // namespace greem
