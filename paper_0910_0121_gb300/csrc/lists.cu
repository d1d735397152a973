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
                               unsigned long long pos0, unsigned long long lim, int lane, uint32_t &nacc)
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
    if (lane == 0) stk[0] = root;
    uint32_t sp = 1;
    bool overflow = false;
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
            const unsigned ab = __ballot_sync(FULL, acc);
            if (acc) {
                const unsigned long long p = pos0 + cnt + __popc(ab & lt);
                const float4 v = __ldg(a.noff + child);
                const float4 e = make_float4(__fadd_rn(__fmul_rn((float)ct.dx, kf), v.x),
                                             __fadd_rn(__fmul_rn((float)ct.dy, kf), v.y),
                                             __fadd_rn(__fmul_rn((float)ct.dz, kf), v.z), v.w);
                if (p < lim) {
                    a.flist[p] = e;
                    if (INDEX)
                        a.ilist[p] = (unsigned long long)child | (1ull << 32) | ((unsigned long long)ct.shc << 33);
                }
            }
            cnt += __popc(ab);
            nacc += __popc(ab);
            const unsigned pb = __ballot_sync(FULL, push);
            if (sp + __popc(pb) > cap) {
                if (lane == 0) atomicOr(&a.st->flags, ST_STACK);
                overflow = true;  // the caller's list is incomplete; the call is retried with a larger stack
                break;
            }
            if (push) stk[sp + __popc(pb & lt)] = child;
            sp += __popc(pb);
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
    __syncthreads();
    if (a.st->flags & ST_NODE_CAP) return;  // the tree was truncated: the call is retried
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
        const uint32_t len = walk_group<INDEX>(a, gr, tb, th, bp, root, stk, octq, page_cur, page_end, lane, nacc);
        const uint32_t padded = (len + 7u) & ~7u;
        if (lane == 0) atomicAdd(&a.st->sum_padded, (unsigned long long)padded);
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
            walk_group<INDEX>(a, gr, tb, th, bp, root, stk, octq, page_cur, page_end, lane, nacc);
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
            atomicAdd(&a.st->sum_len, (unsigned long long)len);
            atomicAdd(&a.st->sum_inter, (unsigned long long)len * gr.count);
        }
        page_cur += padded;
    }
}

void launch_lists(const ListArgs &a, cudaStream_t s, int nsm)
{
    if (a.ilist) k_lists<true><<<nsm * kListBlocksPerSM, kListWarps * 32, 0, s>>>(a);
    else k_lists<false><<<nsm * kListBlocksPerSM, kListWarps * 32, 0, s>>>(a);
    g_launches++;
}

}  // namespace greem
