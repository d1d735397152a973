// S5 Barnes (1990) grouped interaction lists (Sec. 2.2 steps 3 and 5; Sec. 3.1.2).
//
// One warp per group walks its box's tree from the root with a per-warp stack of node
// indices: each step pops up to 32 nodes, one per lane, and each lane decides, in
// this order:
//   prune  -- the node's cell is farther than r_cut from the group's particle box (the
//             box of finest-level cells that holds the group's particles; periodic
//             box-to-box distance), so none of its particles can act (Eq. 2 is 0);
//   accept -- level >= l_min and the opening criterion holds: cell side l and the
//             distance d from the node's cell centre to the nearest point of the group
//             cell satisfy l < theta d; the node enters the list as one particle at its
//             centre of mass (Sec. 3.1.2);
//   leaf   -- an opened leaf puts its particles into the list, each but those whose
//             finest cell passes the prune test (the same integer test at level 21);
//   open   -- the node's children (child table, up to 8) are pushed.
// Every popped node is one the recursive walk visits, so no lane tests a node inside a
// pruned or accepted subtree.  The entries are the same set as the recursive walk's;
// their order within a list is the order of the steps (the debug dump sorts each list
// back into preorder, i.e. by first particle).
// Every test is done in integer units u = L/2^22 against thresholds the host derives
// from the FP64 comparisons (double)S*u*u > r_cut*r_cut and (double)l*l < theta*theta*S,
// so the lists are exact and bit-identical to a sequential FP64 walk.
//
// Entries are written as float4 (x, y, z, m) relative to the group's cell centre in
// eta units (Sec. 3.1.1: positions passed relative to the group centre): the cell
// offset (an exact integer in u, wrapped to the nearest image) times u/eta, plus the
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

// Walks one group's list; writes entries [pos0, pos0+total) clipped at lim; returns
// total.  stk is this warp's stack (a.stack_cap entries); an overflow sets the status.
__device__ uint32_t walk_group(const ListArgs &a, const Group &gr, const int4 tb, const int4 th, const BoxPar &bp,
                               uint32_t root, uint32_t *__restrict__ stk, unsigned long long pos0,
                               unsigned long long lim, int lane)
{
    const unsigned FULL = 0xffffffffu;
    const uint32_t gend = gr.begin + gr.count;
    const long long Tp = bp.T_prune;
    const int lmin = bp.lmin;
    const float kf = bp.k_f;
    const uint32_t cap = a.stack_cap;
    uint32_t cnt = 0;
    if (lane == 0) stk[0] = root;
    uint32_t sp = 1;
    __syncwarp();
    while (sp > 0) {
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
        const bool leaf = (nd.lvl & 256u) != 0;
        const int h = 1 << (kMaxLevel - k);
        int sx, sy, sz;
        const int dx = wrap_delta(2 * (int)nd.ix + h - gr.cx, sx);
        const int dy = wrap_delta(2 * (int)nd.iy + h - gr.cy, sy);
        const int dz = wrap_delta(2 * (int)nd.iz + h - gr.cz, sz);
        const int ax = abs(dx), ay = abs(dy), az = abs(dz);
        const int gx = max(0, abs(dx - tb.x) - h - th.x), gy = max(0, abs(dy - tb.y) - h - th.y),
                  gz = max(0, abs(dz - tb.z) - h - th.z);
        const int ex = max(0, ax - gr.hg), ey = max(0, ay - gr.hg), ez = max(0, az - gr.hg);
        const long long Sg = (long long)gx * gx + (long long)gy * gy + (long long)gz * gz;
        const long long Sd = (long long)ex * ex + (long long)ey * ey + (long long)ez * ez;
        const bool prune = Sg > Tp;
        // an opened leaf whose whole cell lies within r_cut of the particle box keeps every
        // particle (each particle's finest cell is inside the leaf's cell), so its particles
        // skip the per-particle test
        const int fx = max(0, abs(dx - tb.x) + h - th.x), fy = max(0, abs(dy - tb.y) + h - th.y),
                  fz = max(0, abs(dz - tb.z) + h - th.z);
        const bool test_each = (long long)fx * fx + (long long)fy * fy + (long long)fz * fz > Tp;
        const bool accept = !prune && k >= lmin && Sd > bp.A[k];
        const bool open = valid && !prune && !accept && !leaf;
        uint32_t ne = (valid && !prune) ? (accept ? 1u : (leaf ? nd.end - nd.begin : 0u)) : 0u;
        // push the children of opened nodes
        uint4 k0 = make_uint4(kNone, kNone, kNone, kNone), k1 = k0;
        uint32_t nch = 0;
        if (open) {
            const uint4 *kp = reinterpret_cast<const uint4 *>(a.kids + (size_t)m * 8);
            k0 = __ldg(kp);
            k1 = __ldg(kp + 1);
            nch = (k0.x != kNone) + (k0.y != kNone) + (k0.z != kNone) + (k0.w != kNone) + (k1.x != kNone) +
                  (k1.y != kNone) + (k1.z != kNone) + (k1.w != kNone);
        }
        uint32_t csum = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, csum, o);
            if (lane >= o) csum += y;
        }
        const uint32_t ctot = __shfl_sync(FULL, csum, 31);
        if (sp + ctot > cap) {
            if (lane == 0) atomicOr(&a.st->flags, ST_STACK);
            break;  // the caller's list is incomplete; the call is retried with a larger stack
        }
        if (nch) {
            uint32_t *d = stk + sp + (csum - nch);
            const uint32_t kk[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
#pragma unroll
            for (int q = 0; q < 8; q++)
                if ((uint32_t)q < nch) d[q] = kk[q];
        }
        sp += ctot;
        __syncwarp();
        uint32_t isum = ne;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, isum, o);
            if (lane >= o) isum += y;
        }
        const uint32_t off = isum - ne;
        const uint32_t tot = __shfl_sync(FULL, isum, 31);
        if (tot) {
            const float bx = __fmul_rn((float)dx, kf), by = __fmul_rn((float)dy, kf), bz = __fmul_rn((float)dz, kf);
            const uint32_t src = accept ? (m | 0x80000000u) : nd.begin;
            const unsigned shc = shift_code(sx, sy, sz) | ((test_each && !accept) ? 64u : 0u);
            for (uint32_t t0 = 0; t0 < tot; t0 += 32) {
                const uint32_t t = t0 + lane;
                int s = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const uint32_t oc = __shfl_sync(FULL, off, s + step);
                    if (oc <= t) s += step;
                }
                const uint32_t o_s = __shfl_sync(FULL, off, s);
                const uint32_t src_s = __shfl_sync(FULL, src, s);
                const float bx_s = __shfl_sync(FULL, bx, s), by_s = __shfl_sync(FULL, by, s),
                            bz_s = __shfl_sync(FULL, bz, s);
                const unsigned sh_s = __shfl_sync(FULL, shc, s);
                bool keep = false;
                float4 e;
                unsigned long long ie = 0;
                if (t < tot) {
                    float4 v;
                    uint32_t j = kNone;
                    keep = true;
                    if (src_s & 0x80000000u) {
                        const uint32_t nn = src_s & 0x7fffffffu;
                        v = __ldg(a.noff + nn);
                        ie = (unsigned long long)nn | (1ull << 32);
                    } else {
                        j = src_s + (t - o_s);
                        v = __ldg(a.poff + j);
                        ie = (unsigned long long)j;
                    }
                    if (sh_s & 64u) {
                        // the particle's finest cell, in its leaf's image, against the particle box
                        const unsigned long long c = __ldg(a.pcell + j);
                        const int px = 2 * (int)((uint32_t)c & 0x1fffffu) + 1 - gr.cx - tb.x +
                                       ((sh_s & 1u) ? kPeriod : ((sh_s & 2u) ? -kPeriod : 0));
                        const int py = 2 * (int)((uint32_t)(c >> 21) & 0x1fffffu) + 1 - gr.cy - tb.y +
                                       ((sh_s & 4u) ? kPeriod : ((sh_s & 8u) ? -kPeriod : 0));
                        const int pz = 2 * (int)(uint32_t)(c >> 42) + 1 - gr.cz - tb.z +
                                       ((sh_s & 16u) ? kPeriod : ((sh_s & 32u) ? -kPeriod : 0));
                        const int qx = max(0, abs(px) - 1 - th.x), qy = max(0, abs(py) - 1 - th.y),
                                  qz = max(0, abs(pz) - 1 - th.z);
                        keep = (long long)qx * qx + (long long)qy * qy + (long long)qz * qz <= Tp;
                    }
                    e = make_float4(__fadd_rn(bx_s, v.x), __fadd_rn(by_s, v.y), __fadd_rn(bz_s, v.z), v.w);
                    if (j >= gr.begin && j < gend) a.irel[j] = e;
                }
                const unsigned kb = __ballot_sync(FULL, keep);
                if (keep) {
                    const unsigned long long p = pos0 + cnt + __popc(kb & ((1u << lane) - 1u));
                    if (p < lim) {
                        a.flist[p] = e;
                        if (a.ilist) a.ilist[p] = ie | ((unsigned long long)(sh_s & 63u) << 33);
                    }
                }
                cnt += __popc(kb);
            }
        }
    }
    __syncwarp();
    return cnt;
}

__global__ void __launch_bounds__(kListWarps * 32, kListBlocksPerSM) k_lists(ListArgs a)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
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
        const uint32_t len = walk_group(a, gr, tb, th, bp, root, stk, page_cur, page_end, lane);
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
            walk_group(a, gr, tb, th, bp, root, stk, page_cur, page_end, lane);
        }
        for (uint32_t t = len + lane; t < padded; t += 32) {
            a.flist[page_cur + t] = make_float4(16.f, 16.f, 16.f, 0.f);
            if (a.ilist) a.ilist[page_cur + t] = ~0ull;
        }
        if (lane == 0) {
            a.loff[g] = page_cur;
            a.llen[g] = padded;
            a.lraw[g] = len;
            atomicAdd(&a.st->sum_len, (unsigned long long)len);
            atomicAdd(&a.st->sum_inter, (unsigned long long)len * gr.count);
        }
        page_cur += padded;
    }
}

void launch_lists(const ListArgs &a, cudaStream_t s, int nsm)
{
    k_lists<<<nsm * kListBlocksPerSM, kListWarps * 32, 0, s>>>(a);
    g_launches++;
}

}  // namespace greem
