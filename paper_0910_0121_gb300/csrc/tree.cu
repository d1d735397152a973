// S3 octree + monopole moments and S4 groups, built from the sorted Morton keys.
//
// The tree is the paper's local tree (Sec. 2.2 step 2) with the N_leaf stop rule
// (Sec. 3.1.2: a node holding fewer than N_leaf particles is not subdivided).  Levels
// above l_min are always split so that every accepted node and every group is small
// enough for a single periodic image shift per node.
//
// Construction without recursion.  Let d_i be the first level at which key i differs
// from key i-1 (0 for the first particle of a box, 22 for equal keys): the cells of
// levels d_i..21 that contain particle i start at i.  Let K_i be the level of the leaf
// containing i: the deepest level whose parent cell holds at least N_leaf particles
// (or lies above l_min), capped at 21.  A level-j cell holds >= N_leaf particles iff
// some window of N_leaf consecutive sorted particles containing i shares its level-j
// prefix, so K_i comes from a sliding maximum over such windows.  Particle i then owns
// the nodes (i, d_i) ... (i, K_i); an exclusive scan of the ownership counts numbers
// the nodes in DFS preorder, because preorder is the order of (begin, level).
#include <algorithm>

#include "common.cuh"

namespace greem {

__device__ __forceinline__ int lcp_level(uint64_t a, uint64_t b)
{
    uint64_t x = a ^ b;
    if (x == 0) return kMaxLevel;
    return (__clzll((long long)x) - 1) / 3;  // bit 63 is zero in both keys
}

__device__ __forceinline__ uint32_t compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

// Window LCPs of a block: w[t] = lcp_level(keys[t], keys[t + N_leaf - 1]) for the windows
// t = i0 - kPrepHalo ... i0 + 255 that stay inside their box (-1 otherwise), computed once
// and shared by the N_leaf particles each window covers.
constexpr int kPrepHalo = 64;

__global__ void __launch_bounds__(256) k_tree_prep(const uint64_t *__restrict__ keys, uint32_t N,
                                                   const uint32_t *__restrict__ box_off, int nbox,
                                                   const BoxPar *__restrict__ bps, uint8_t *__restrict__ d8,
                                                   uint8_t *__restrict__ K8, uint32_t *__restrict__ own)
{
    __shared__ int8_t ws[256 + kPrepHalo];
    const long long i0 = (long long)blockIdx.x * 256;
    for (int k = threadIdx.x; k < 256 + kPrepHalo; k += 256) {
        const long long t = i0 - kPrepHalo + k;
        int w = -1;
        if (t >= 0 && t < (long long)N) {
            const int bt = box_of((uint32_t)t, box_off, nbox);
            const int nl = bps[bt].n_leaf;
            if (nl <= kPrepHalo + 1 && t + nl - 1 < (long long)box_off[bt + 1])
                w = lcp_level(keys[t], keys[t + nl - 1]);
        }
        ws[k] = (int8_t)w;
    }
    __syncthreads();
    const uint32_t i = (uint32_t)i0 + threadIdx.x;
    if (i >= N) return;
    const int b = box_of(i, box_off, nbox);
    const long long o = box_off[b], e = box_off[b + 1];
    const int nl = bps[b].n_leaf, lmin = bps[b].lmin;
    const uint64_t ki = keys[i];
    int d = (i == (uint32_t)o) ? 0 : lcp_level(keys[i - 1], ki) + 1;
    int J = -1;
    long long tlo = (long long)i - nl + 1;
    if (tlo < o) tlo = o;
    long long thi = e - nl;
    if (thi > (long long)i) thi = i;
    if (nl <= kPrepHalo + 1) {
        for (long long t = tlo; t <= thi; t++) J = max(J, (int)ws[t - i0 + kPrepHalo]);
    } else {
        for (long long t = tlo; t <= thi; t++) {
            int w = lcp_level(keys[t], keys[t + nl - 1]);
            J = w > J ? w : J;
        }
    }
    int K = J + 1;
    K = K < lmin ? lmin : K;
    K = K > kMaxLevel ? kMaxLevel : K;
    d8[i] = (uint8_t)d;
    K8[i] = (uint8_t)K;
    own[i] = d <= K ? (uint32_t)(K - d + 1) : 0u;
}

void launch_tree_prep(const uint64_t *keys, uint32_t N, const uint32_t *box_off, int nbox, const BoxPar *bps,
                      uint8_t *d8, uint8_t *K8, uint32_t *own, cudaStream_t s)
{
    k_tree_prep<<<(N + 255) / 256, 256, 0, s>>>(keys, N, box_off, nbox, bps, d8, K8, own);
    g_launches++;
}

// End of the level-k cell that contains sorted particle i (k >= 1): the first index
// j in (lo, e] whose level-k prefix differs, searched by galloping from lo, where lo
// is known to share the prefix.
__device__ __forceinline__ uint32_t cell_end(const uint64_t *__restrict__ keys, uint32_t lo, uint32_t e,
                                             uint64_t pfx, int shift)
{
    uint32_t step = 1, hi;
    for (;;) {
        uint32_t j = lo + step;
        if (j >= e) { hi = e; break; }
        if ((keys[j] >> shift) != pfx) { hi = j; break; }
        lo = j;
        step <<= 1;
    }
    while (hi - lo > 1) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if ((keys[mid] >> shift) == pfx) lo = mid; else hi = mid;
    }
    return hi;
}

// The nodes owned by sorted particle i (own > 0 of them, numbered from b0).
__device__ __forceinline__ void fill_nodes(const uint64_t *__restrict__ keys, uint32_t i, uint32_t b0,
                                           const uint32_t *__restrict__ box_off, int nbox,
                                           const uint8_t *__restrict__ d8, const uint8_t *__restrict__ K8,
                                           const uint32_t *__restrict__ base, Node *__restrict__ nodes,
                                           uint32_t node_cap)
{
    const int b = box_of(i, box_off, nbox);
    const uint32_t e = box_off[b + 1];
    const int d = d8[i], K = K8[i];
    const uint64_t key = keys[i];
    const uint32_t cx = compact3(key >> 2), cy = compact3(key >> 1), cz = compact3(key);
    uint32_t end = i + 1;
    for (int k = K; k >= d; k--) {
        const uint32_t n = b0 + (uint32_t)(k - d);
        if (k == 0) {
            end = e;
        } else {
            const int shift = 3 * (kMaxLevel - k);
            end = cell_end(keys, end - 1, e, key >> shift, shift);
        }
        if (n < node_cap) {
            const uint32_t mask = k == 0 ? 0u : ~((1u << (kMaxLevel - k)) - 1u);
            Node nd;
            nd.ix = cx & mask;
            nd.iy = cy & mask;
            nd.iz = cz & mask;
            nd.lvl = (uint32_t)k | (k == K ? 256u : 0u);
            nd.begin = i;
            nd.end = end;
            nd.skip = base[end];
            nd.parent = kNone;
            nodes[n] = nd;
        }
    }
}

// About one particle in five owns nodes.  Each warp queues the owners among its 32
// particles in shared memory and fills nodes 32 owners at a time, so that every lane of
// a filling warp has an owner's galloping searches to run.
__global__ void __launch_bounds__(256) k_tree_fill(const uint64_t *__restrict__ keys, uint32_t N,
                                                   const uint32_t *__restrict__ box_off, int nbox,
                                                   const uint8_t *__restrict__ d8, const uint8_t *__restrict__ K8,
                                                   const uint32_t *__restrict__ base, Node *__restrict__ nodes,
                                                   uint32_t node_cap, DevStatus *st)
{
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ uint32_t queue[8][64];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t *q = queue[w];
    uint32_t qn = 0;  // queued owners (the same in every lane)
    const uint32_t nchunks = (N + 31) / 32, nwarps = gridDim.x * 8;
    for (uint32_t ch = blockIdx.x * 8 + (uint32_t)w; ch < nchunks; ch += nwarps) {
        const uint32_t i = ch * 32 + (uint32_t)lane;
        bool owner = false;
        if (i < N) {
            owner = base[i + 1] > base[i];
            if (i == N - 1 && base[N] > node_cap) atomicOr(&st->flags, ST_NODE_CAP);
        }
        const unsigned m = __ballot_sync(FULL, owner);
        if (owner) q[qn + __popc(m & lt)] = i;
        qn += __popc(m);
        __syncwarp();
        if (qn >= 32) {
            const uint32_t j = q[lane];
            fill_nodes(keys, j, base[j], box_off, nbox, d8, K8, base, nodes, node_cap);
            __syncwarp();
            if ((uint32_t)lane < qn - 32) q[lane] = q[32 + lane];  // at most 31 left, from slots 32..62
            __syncwarp();
            qn -= 32;
        }
    }
    if ((uint32_t)lane < qn) {
        const uint32_t j = q[lane];
        fill_nodes(keys, j, base[j], box_off, nbox, d8, K8, base, nodes, node_cap);
    }
}

void launch_tree_fill(const uint64_t *keys, uint32_t N, const uint32_t *box_off, int nbox, const uint8_t *d8,
                      const uint8_t *K8, const uint32_t *base, Node *nodes, uint32_t node_cap, DevStatus *st,
                      cudaStream_t s, int nsm)
{
    const unsigned grid = (unsigned)std::min<size_t>((N + 255) / 256, (size_t)nsm * 8);
    k_tree_fill<<<grid, 256, 0, s>>>(keys, N, box_off, nbox, d8, K8, base, nodes, node_cap, st);
    g_launches++;
}

__device__ __forceinline__ uint32_t node_count(const uint32_t *n_nodes, uint32_t cap)
{
    uint32_t n = *n_nodes;
    return n < cap ? n : cap;
}

// Parent links, child counts, the child table (up to 8 children per internal node,
// unused slots kNone) and each node's child-octant mask (bits 16-23 of lvl; octant =
// x<<2 | y<<1 | z of the child's cell within the parent's): the children of an internal
// node p are p+1 and then the skip chain while it stays inside p's particle range, in
// Morton order, so slot q holds the child in the octant of the mask's (q+1)-th set bit.
__global__ void __launch_bounds__(256) k_tree_links(Node *__restrict__ nodes, const uint32_t *__restrict__ n_nodes,
                                                    uint32_t node_cap, uint8_t *__restrict__ nchild,
                                                    uint32_t *__restrict__ kids)
{
    const uint32_t nn = node_count(n_nodes, node_cap);
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += gridDim.x * blockDim.x) {
        const Node np = nodes[p];
        uint32_t slot[8];
#pragma unroll
        for (int k = 0; k < 8; k++) slot[k] = kNone;
        uint32_t cnt = 0, mask = 0;
        if (!(np.lvl & 256u)) {
            const int sh = kMaxLevel - 1 - (int)(np.lvl & 255u);  // child side in finest cells = 1 << sh
            uint32_t c = p + 1;
            while (c < nn && nodes[c].begin < np.end && cnt < 8) {
                const Node nc = nodes[c];
                nodes[c].parent = p;
                mask |= 1u << ((((nc.ix >> sh) & 1u) << 2) | (((nc.iy >> sh) & 1u) << 1) | ((nc.iz >> sh) & 1u));
#pragma unroll
                for (int k = 0; k < 8; k++)
                    if (k == (int)cnt) slot[k] = c;
                cnt++;
                c = nc.skip;
            }
            nodes[p].lvl = np.lvl | (mask << 16);
        }
        nchild[p] = (uint8_t)cnt;
        uint4 *kp = reinterpret_cast<uint4 *>(kids + (size_t)p * 8);
        kp[0] = make_uint4(slot[0], slot[1], slot[2], slot[3]);
        kp[1] = make_uint4(slot[4], slot[5], slot[6], slot[7]);
    }
}

void launch_tree_links(Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, uint8_t *nchild, uint32_t *kids,
                       cudaStream_t s, int nsm)
{
    k_tree_links<<<nsm * 8, 256, 0, s>>>(nodes, n_nodes, node_cap, nchild, kids);
    g_launches++;
}

// Monopole moments (Sec. 3.1.2, centre-of-mass approximation), bottom up.  Leaves sum
// their particles in FP64 by tiles of consecutive particles (k_moments_leaf_tiled below:
// coalesced loads, and within a tile the leaves taken in order of particle count, so the
// lanes of a warp loop over equally many particles: an FP64 warp instruction costs the
// same with idle lanes, and FP64 issue is expensive on this GPU).  Internal nodes are
// bucketed by level and follow level by level, deepest first, each summing its
// children's raw moments in child order.  Every sum has a fixed order, so the result
// does not depend on scheduling.
//
// lvl[0..64): nodes per bucket, lvl[64..128): bucket start, lvl[128..192): cursor.
constexpr int kLeafBucket = 32;

__device__ __forceinline__ uint32_t node_bucket(const Node &nd)
{
    return (nd.lvl & 256u) ? kLeafBucket + min(nd.end - nd.begin, 31u) : (nd.lvl & 255u);
}

__global__ void __launch_bounds__(256) k_node_buckets(const Node *__restrict__ nodes,
                                                      const uint32_t *__restrict__ n_nodes, uint32_t node_cap,
                                                      uint32_t *__restrict__ lvl)
{
    __shared__ uint32_t cnt[64];
    if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t nn = node_count(n_nodes, node_cap);
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < nn) {
        const Node nd = nodes[n];
        if (!(nd.lvl & 256u)) atomicAdd(&cnt[node_bucket(nd)], 1u);  // leaves are summed by tiles
    }
    __syncthreads();
    if (threadIdx.x < 64 && cnt[threadIdx.x]) atomicAdd(&lvl[threadIdx.x], cnt[threadIdx.x]);
}

__global__ void k_level_scan(uint32_t *lvl)
{
    const uint32_t lane = threadIdx.x;
    const uint32_t v0 = lvl[lane], v1 = lvl[32 + lane];
    uint32_t x0 = v0, x1 = v1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, x1, o);
        if (lane >= (uint32_t)o) {
            x0 += y0;
            x1 += y1;
        }
    }
    const uint32_t tot0 = __shfl_sync(0xffffffffu, x0, 31);
    lvl[64 + lane] = lvl[128 + lane] = x0 - v0;
    lvl[96 + lane] = lvl[160 + lane] = tot0 + x1 - v1;
}

// Places every node in its bucket: a slot within the block from a shared-memory counter,
// then one global atomic per bucket and block.  The order within a bucket is free (its
// nodes are summed independently).
__global__ void __launch_bounds__(256) k_level_scatter(const Node *__restrict__ nodes,
                                                       const uint32_t *__restrict__ n_nodes, uint32_t node_cap,
                                                       uint32_t *__restrict__ lvl, uint32_t *__restrict__ inodes)
{
    __shared__ uint32_t cnt[64], base[64];
    if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t nn = node_count(n_nodes, node_cap);
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t key = 0, slot = 0;
    bool inner = false;
    if (n < nn) {
        const Node nd = nodes[n];
        inner = !(nd.lvl & 256u);  // leaves are summed by tiles
        if (inner) {
            key = node_bucket(nd);
            slot = atomicAdd(&cnt[key], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < 64 && cnt[threadIdx.x]) base[threadIdx.x] = atomicAdd(&lvl[128 + threadIdx.x], cnt[threadIdx.x]);
    __syncthreads();
    if (inner) inodes[base[key] + slot] = n;
}

// Leaf moments by tiles of consecutive particles: a block takes the leaves that start in
// its tile of kLeafTile sorted particles (the deepest node a particle owns is a leaf, so
// particle i starts leaf base[i+1] - 1 when it owns any node), stages the tile's
// particles and a halo in shared memory with coalesced loads, and orders its leaves by
// particle count, so that the lanes of a warp loop equally often (an FP64 warp
// instruction costs the same with idle lanes).  Each leaf sums its particles in sorted
// order, as a thread alone would.  Leaves reaching past the halo read the rest from
// global memory.
constexpr int kLeafTile = 1024;
constexpr int kLeafHalo = 64;

__global__ void __launch_bounds__(256) k_moments_leaf_tiled(const Node *__restrict__ nodes,
                                                            const uint32_t *__restrict__ n_nodes, uint32_t node_cap,
                                                            const uint32_t *__restrict__ base, uint32_t N,
                                                            const double *__restrict__ xs,
                                                            const double *__restrict__ ys,
                                                            const double *__restrict__ zs,
                                                            const float *__restrict__ ms, Dbl4 *__restrict__ raw)
{
    __shared__ double sx_[kLeafTile + kLeafHalo], sy_[kLeafTile + kLeafHalo], sz_[kLeafTile + kLeafHalo];
    __shared__ float sm_[kLeafTile + kLeafHalo];
    __shared__ uint32_t leaf_n[kLeafTile], leaf_b[kLeafTile], leaf_e[kLeafTile], order[kLeafTile];
    __shared__ uint32_t cnt[33], start[33], nleaf;
    const uint32_t nn = node_count(n_nodes, node_cap);
    const uint32_t p0 = blockIdx.x * kLeafTile;
    const uint32_t pe = min(N, p0 + kLeafTile + kLeafHalo);
    const int tid = threadIdx.x;
    if (tid < 33) cnt[tid] = 0;
    if (tid == 0) nleaf = 0;
    for (uint32_t q = tid; q < pe - p0; q += blockDim.x) {
        sx_[q] = xs[p0 + q];
        sy_[q] = ys[p0 + q];
        sz_[q] = zs[p0 + q];
        sm_[q] = ms[p0 + q];
    }
    __syncthreads();
    // the leaves that start in the tile
    const uint32_t pt = min(N, p0 + kLeafTile);
    for (uint32_t i = p0 + tid; i < pt; i += blockDim.x) {
        const uint32_t o0 = base[i], o1 = base[i + 1];
        if (o1 == o0) continue;
        const uint32_t n = o1 - 1;
        if (n >= nn) continue;  // a truncated tree: the call is retried
        const uint32_t e = nodes[n].end;
        const uint32_t slot = atomicAdd(&nleaf, 1u);
        leaf_n[slot] = n;
        leaf_b[slot] = i;
        leaf_e[slot] = e;
        atomicAdd(&cnt[min(e - i, 32u)], 1u);
    }
    __syncthreads();
    if (tid < 32) {  // bucket starts by particle count (1..31, then 32 and more)
        const uint32_t v = cnt[tid + 1];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (tid >= o) x += y;
        }
        start[tid + 1] = x - v;
    }
    __syncthreads();
    const uint32_t L = nleaf;
    for (uint32_t k = tid; k < L; k += blockDim.x) order[atomicAdd(&start[min(leaf_e[k] - leaf_b[k], 32u)], 1u)] = k;
    __syncthreads();
    for (uint32_t q = tid; q < L; q += blockDim.x) {
        const uint32_t k = order[q];
        const uint32_t b = leaf_b[k], e = leaf_e[k];
        double M = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
        for (uint32_t j = b; j < e; j++) {
            double m, x, y, z;
            if (j < pe) {
                m = (double)sm_[j - p0];
                x = sx_[j - p0];
                y = sy_[j - p0];
                z = sz_[j - p0];
            } else {
                m = (double)ms[j];
                x = xs[j];
                y = ys[j];
                z = zs[j];
            }
            M += m;
            ax = fma(m, x, ax);
            ay = fma(m, y, ay);
            az = fma(m, z, az);
        }
        raw[leaf_n[k]] = make_dbl4(ax, ay, az, M);
    }
}

__global__ void __launch_bounds__(256) k_moments_level(int level, const uint32_t *__restrict__ lvl,
                                                       const uint32_t *__restrict__ inodes,
                                                       const uint32_t *__restrict__ kids, Dbl4 *__restrict__ raw)
{
    const uint32_t b = lvl[64 + level], e = b + lvl[level];
    for (uint32_t i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) {
        const uint32_t p = inodes[i];
        const uint4 *kp = reinterpret_cast<const uint4 *>(kids + (size_t)p * 8);
        const uint4 k0 = kp[0], k1 = kp[1];
        const uint32_t kk[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
        Dbl4 a = make_dbl4(0.0, 0.0, 0.0, 0.0);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            if (kk[q] == kNone) break;
            const Dbl4 r = raw[kk[q]];
            a.x += r.x;
            a.y += r.y;
            a.z += r.z;
            a.w += r.w;
        }
        raw[p] = a;
    }
}

void launch_moments(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const uint32_t *kids,
                    const uint32_t *base, uint32_t N, const double *xs, const double *ys, const double *zs,
                    const float *ms, Dbl4 *raw, uint32_t *lvl, uint32_t *inodes, cudaStream_t s, int nsm)
{
    (void)nsm;
    cudaMemsetAsync(lvl, 0, 192 * sizeof(uint32_t), s);
    const unsigned grid = (node_cap + 255) / 256;
    k_node_buckets<<<grid, 256, 0, s>>>(nodes, n_nodes, node_cap, lvl);
    k_level_scan<<<1, 32, 0, s>>>(lvl);
    k_level_scatter<<<grid, 256, 0, s>>>(nodes, n_nodes, node_cap, lvl, inodes);
    k_moments_leaf_tiled<<<(N + kLeafTile - 1) / kLeafTile, 256, 0, s>>>(nodes, n_nodes, node_cap, base, N, xs, ys,
                                                                       zs, ms, raw);
    g_launches += 4;
    for (int level = kMaxLevel - 1; level >= 0; level--) {
        k_moments_level<<<nsm * 4, 256, 0, s>>>(level, lvl, inodes, kids, raw);
        g_launches++;
    }
}

// Second moments about the COM (the second-order terms of Sec. 4.1), FP32 in r_cut^2 units,
// as two float4 per node: (xx, yy, zz, xy), (xz, yz, (xx+yy+zz)/2, 0).  A leaf sums
// m (p - c)(p - c)^T over its particles, p the particle's offset from the leaf's cell
// centre and c the COM's (both already in r_cut units).  An internal node adds its
// children's moments moved to its own COM (parallel axes): Q_c + M_c d_c d_c^T, d_c =
// child COM - node COM, from the exact cell-centre difference and the COM offsets.
__device__ __forceinline__ void quad_store(float4 *__restrict__ quad, uint32_t n, const float q[6])
{
    quad[2 * (size_t)n] = make_float4(q[0], q[1], q[2], q[3]);
    quad[2 * (size_t)n + 1] = make_float4(q[4], q[5], 0.5f * (q[0] + q[1] + q[2]), 0.f);
}

__global__ void __launch_bounds__(256) k_quad_leaf(const Node *__restrict__ nodes, const uint32_t *__restrict__ n_nodes,
                                                   uint32_t node_cap, const float4 *__restrict__ poff,
                                                   const float4 *__restrict__ noff, float4 *__restrict__ quad)
{
    const uint32_t nn = node_count(n_nodes, node_cap);
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += gridDim.x * blockDim.x) {
        const Node nd = nodes[n];
        if (!(nd.lvl & 256u)) continue;
        const float4 c = noff[n];
        float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (uint32_t j = nd.begin; j < nd.end; j++) {
            const float4 p = poff[j];
            const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
            const float mx = p.w * dx, my = p.w * dy, mz = p.w * dz;
            q[0] = fmaf(mx, dx, q[0]);
            q[1] = fmaf(my, dy, q[1]);
            q[2] = fmaf(mz, dz, q[2]);
            q[3] = fmaf(mx, dy, q[3]);
            q[4] = fmaf(mx, dz, q[4]);
            q[5] = fmaf(my, dz, q[5]);
        }
        quad_store(quad, n, q);
    }
}

__global__ void __launch_bounds__(256) k_quad_level(int level, const uint32_t *__restrict__ lvl,
                                                    const uint32_t *__restrict__ inodes,
                                                    const Node *__restrict__ nodes, const uint32_t *__restrict__ kids,
                                                    const float4 *__restrict__ noff,
                                                    const uint32_t *__restrict__ box_off, int nbox,
                                                    const BoxPar *__restrict__ bps, float4 *__restrict__ quad)
{
    const uint32_t b = lvl[64 + level], e = b + lvl[level];
    for (uint32_t i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) {
        const uint32_t p = inodes[i];
        const Node np = nodes[p];
        const float kf = bps[box_of(np.begin, box_off, nbox)].k_f;
        const int hp = 1 << (kMaxLevel - level);
        const float4 cp = noff[p];
        float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const uint4 *kp = reinterpret_cast<const uint4 *>(kids + (size_t)p * 8);
        const uint4 k0 = kp[0], k1 = kp[1];
        const uint32_t kk[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
#pragma unroll
        for (int t = 0; t < 8; t++) {
            const uint32_t c = kk[t];
            if (c == kNone) break;
            const Node nc = nodes[c];
            const int hc = hp >> 1;
            const float4 cc = noff[c];
            // child COM - node COM: cell-centre difference (exact integer in u) and COM offsets
            const float dx = fmaf((float)(2 * ((int)nc.ix - (int)np.ix) + hc - hp), kf, cc.x - cp.x);
            const float dy = fmaf((float)(2 * ((int)nc.iy - (int)np.iy) + hc - hp), kf, cc.y - cp.y);
            const float dz = fmaf((float)(2 * ((int)nc.iz - (int)np.iz) + hc - hp), kf, cc.z - cp.z);
            const float4 q0 = quad[2 * (size_t)c], q1 = quad[2 * (size_t)c + 1];
            const float mx = cc.w * dx, my = cc.w * dy, mz = cc.w * dz;
            q[0] += fmaf(mx, dx, q0.x);
            q[1] += fmaf(my, dy, q0.y);
            q[2] += fmaf(mz, dz, q0.z);
            q[3] += fmaf(mx, dy, q0.w);
            q[4] += fmaf(mx, dz, q1.x);
            q[5] += fmaf(my, dz, q1.y);
        }
        quad_store(quad, p, q);
    }
}

void launch_quadrupoles(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const uint32_t *kids,
                        const float4 *poff, const float4 *noff, const uint32_t *lvl, const uint32_t *inodes,
                        const uint32_t *box_off, int nbox, const BoxPar *bps, float4 *quad, cudaStream_t s, int nsm)
{
    k_quad_leaf<<<nsm * 8, 256, 0, s>>>(nodes, n_nodes, node_cap, poff, noff, quad);
    g_launches++;
    for (int level = kMaxLevel - 1; level >= 0; level--) {
        k_quad_level<<<nsm * 4, 256, 0, s>>>(level, lvl, inodes, nodes, kids, noff, box_off, nbox, bps, quad);
        g_launches++;
    }
}

// Each particle's offset from the centre of its leaf cell (level K_i) in r_cut units: the
// FP64 subtraction is done once per particle, then rounded to FP32 for the list builder.
// The general-L form is a real call so that it is not predicated into the integer form's
// lanes (FP64 instructions are slow on this GPU).
static __device__ __noinline__ float4 leaf_offset_fp64(double x, double y, double z, float m, uint32_t cx,
                                                       uint32_t cy, uint32_t cz, double u, double ie)
{
    const double cxa = __dmul_rn((double)cx, u), cya = __dmul_rn((double)cy, u), cza = __dmul_rn((double)cz, u);
    return make_float4((float)__dmul_rn(__dsub_rn(x, cxa), ie), (float)__dmul_rn(__dsub_rn(y, cya), ie),
                       (float)__dmul_rn(__dsub_rn(z, cza), ie), m);
}

__global__ void __launch_bounds__(256) k_leaf_offsets(const uint64_t *__restrict__ keys, const uint8_t *__restrict__ K8,
                                                      uint32_t N, const uint32_t *__restrict__ box_off, int nbox,
                                                      const BoxPar *__restrict__ bps, const double *__restrict__ xs,
                                                      const double *__restrict__ ys, const double *__restrict__ zs,
                                                      const float *__restrict__ ms, float4 *__restrict__ poff,
                                                      unsigned long long *__restrict__ pcell)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const BoxPar &bp = bps[box_of(i, box_off, nbox)];
    const int k = K8[i];
    const uint32_t h = 1u << (kMaxLevel - k);
    const uint32_t mask = ~(h - 1u);
    const uint64_t key = keys[i];
    const uint32_t fx = compact3(key >> 2), fy = compact3(key >> 1), fz = compact3(key);
    pcell[i] = (unsigned long long)fx | ((unsigned long long)fy << 21) | ((unsigned long long)fz << 42);
    const uint32_t cx = 2u * (fx & mask) + h, cy = 2u * (fy & mask) + h, cz = 2u * (fz & mask) + h;
    if (bp.pow2_e != kNotPow2) {
        // integer offsets in units of L/2^52 (centre = c_u * 2^30), one rounding to FP32
        const int e = bp.pow2_e;
        const float s = bp.k52_f;
        poff[i] = make_float4(__ll2float_rn(fixed52(xs[i], e) - ((long long)cx << 30)) * s,
                              __ll2float_rn(fixed52(ys[i], e) - ((long long)cy << 30)) * s,
                              __ll2float_rn(fixed52(zs[i], e) - ((long long)cz << 30)) * s, ms[i]);
        return;
    }
    poff[i] = leaf_offset_fp64(xs[i], ys[i], zs[i], ms[i], cx, cy, cz, bp.u, bp.inv_rc);
}

void launch_leaf_offsets(const uint64_t *keys, const uint8_t *K8, uint32_t N, const uint32_t *box_off, int nbox,
                         const BoxPar *bps, const double *xs, const double *ys, const double *zs, const float *ms,
                         float4 *poff, unsigned long long *pcell, cudaStream_t s)
{
    k_leaf_offsets<<<(N + 255) / 256, 256, 0, s>>>(keys, K8, N, box_off, nbox, bps, xs, ys, zs, ms, poff, pcell);
    g_launches++;
}

// Per leaf, the box of its particles' finest cells, rounded outward to 1/256 of the leaf
// cell's side: per axis the first and last occupied slot, slots of q = max(1, s/256)
// finest cells (s = the cell side in finest cells), 8 bits each, packed as
// x_lo | x_hi << 8 | y_lo << 16 | y_hi << 24 | z_lo << 32 | z_hi << 40.  The list builder
// drops an opened leaf whose box lies beyond r_cut of the group and skips the
// per-particle test of one whose box lies within it: both decisions are those of every
// particle's own test, so the lists are unchanged.
__global__ void __launch_bounds__(256) k_leaf_boxes(const Node *__restrict__ nodes, const uint32_t *__restrict__ n_nodes,
                                                    uint32_t node_cap, const unsigned long long *__restrict__ pcell,
                                                    unsigned long long *__restrict__ lbox)
{
    const uint32_t nn = node_count(n_nodes, node_cap);
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += gridDim.x * blockDim.x) {
        const Node nd = nodes[n];
        if (!(nd.lvl & 256u)) continue;
        const int k = (int)(nd.lvl & 255u);
        const uint32_t sh = (kMaxLevel - k) > 8 ? (uint32_t)(kMaxLevel - k - 8) : 0u;  // q = 2^sh
        uint32_t lo[3] = {255u, 255u, 255u}, hi[3] = {0u, 0u, 0u};
        const uint32_t org[3] = {nd.ix, nd.iy, nd.iz};
        for (uint32_t j = nd.begin; j < nd.end; j++) {
            const unsigned long long c = pcell[j];
            const uint32_t f[3] = {(uint32_t)c & 0x1fffffu, (uint32_t)(c >> 21) & 0x1fffffu, (uint32_t)(c >> 42)};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const uint32_t slot = (f[a] - org[a]) >> sh;
                lo[a] = min(lo[a], slot);
                hi[a] = max(hi[a], slot);
            }
        }
        lbox[n] = (unsigned long long)lo[0] | ((unsigned long long)hi[0] << 8) | ((unsigned long long)lo[1] << 16) |
                  ((unsigned long long)hi[1] << 24) | ((unsigned long long)lo[2] << 32) |
                  ((unsigned long long)hi[2] << 40);
    }
}

void launch_leaf_boxes(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap,
                       const unsigned long long *pcell, unsigned long long *lbox, cudaStream_t s, int nsm)
{
    k_leaf_boxes<<<nsm * 8, 256, 0, s>>>(nodes, n_nodes, node_cap, pcell, lbox);
    g_launches++;
}

// COM offset from the cell centre for a general L (FP64), as a real call (see
// leaf_offset_fp64).
static __device__ __noinline__ float4 node_offset_fp64(double cx, double cy, double cz, float m, uint32_t ux,
                                                       uint32_t uy, uint32_t uz, double u, double ie)
{
    const double cxa = __dmul_rn((double)ux, u), cya = __dmul_rn((double)uy, u), cza = __dmul_rn((double)uz, u);
    return make_float4((float)__dmul_rn(__dsub_rn(cx, cxa), ie), (float)__dmul_rn(__dsub_rn(cy, cya), ie),
                       (float)__dmul_rn(__dsub_rn(cz, cza), ie), m);
}

// COM = S/M (the cell centre for a massless node), and the COM's offset from the node's
// cell centre in r_cut units for the list builder.
__global__ void __launch_bounds__(256) k_node_finish(const Node *__restrict__ nodes,
                                                     const uint32_t *__restrict__ n_nodes, uint32_t node_cap,
                                                     const Dbl4 *__restrict__ raw,
                                                     const uint32_t *__restrict__ box_off, int nbox,
                                                     const BoxPar *__restrict__ bps, Dbl4 *__restrict__ mom64,
                                                     float4 *__restrict__ noff)
{
    const uint32_t nn = node_count(n_nodes, node_cap);
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += gridDim.x * blockDim.x) {
        const Node nd = nodes[n];
        const BoxPar &bp = bps[box_of(nd.begin, box_off, nbox)];
        const int k = nd.lvl & 255u;
        const uint32_t h = 1u << (kMaxLevel - k);
        const Dbl4 r = raw[n];
        double cx, cy, cz;
        if (r.w > 0.0) {
            const double inv = 1.0 / r.w;
            cx = r.x * inv;
            cy = r.y * inv;
            cz = r.z * inv;
        } else {
            // no mass: the cell centre stands in for the centre of mass
            cx = __dmul_rn((double)(2u * nd.ix + h), bp.u);
            cy = __dmul_rn((double)(2u * nd.iy + h), bp.u);
            cz = __dmul_rn((double)(2u * nd.iz + h), bp.u);
        }
        mom64[n] = make_dbl4(cx, cy, cz, r.w);
        if (bp.pow2_e != kNotPow2) {
            const int e = bp.pow2_e;
            const float s = bp.k52_f;
            const long long sh = 30;
            noff[n] = make_float4(__ll2float_rn(fixed52(cx, e) - ((long long)(2u * nd.ix + h) << sh)) * s,
                                  __ll2float_rn(fixed52(cy, e) - ((long long)(2u * nd.iy + h) << sh)) * s,
                                  __ll2float_rn(fixed52(cz, e) - ((long long)(2u * nd.iz + h) << sh)) * s, (float)r.w);
        } else {
            noff[n] = node_offset_fp64(cx, cy, cz, (float)r.w, 2u * nd.ix + h, 2u * nd.iy + h, 2u * nd.iz + h, bp.u,
                                       bp.inv_rc);
        }
    }
}

void launch_node_finish(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const Dbl4 *raw,
                        const uint32_t *box_off, int nbox, const BoxPar *bps, Dbl4 *mom64, float4 *noff,
                        cudaStream_t s, int nsm)
{
    k_node_finish<<<nsm * 8, 256, 0, s>>>(nodes, n_nodes, node_cap, raw, box_off, nbox, bps, mom64, noff);
    g_launches++;
}

// S4 groups (Sec. 2.2 step 5, Sec. 3.1.2 N_crit): a node is a group when it is at level
// >= l_min and holds at most n_crit particles (or is a leaf), and its parent is not.
__device__ __forceinline__ bool group_cond(const Node &nd, const BoxPar &bp)
{
    const int k = nd.lvl & 255u;
    return k >= bp.lmin && ((int)(nd.end - nd.begin) <= bp.n_crit || (nd.lvl & 256u));
}

__global__ void __launch_bounds__(256) k_group_flags(const Node *__restrict__ nodes,
                                                     const uint32_t *__restrict__ n_nodes, uint32_t node_cap,
                                                     const uint32_t *__restrict__ box_off, int nbox,
                                                     const BoxPar *__restrict__ bps, uint32_t *__restrict__ flag)
{
    const uint32_t nn = node_count(n_nodes, node_cap);
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < node_cap; n += gridDim.x * blockDim.x) {
        uint32_t f = 0;
        if (n < nn) {
            const Node nd = nodes[n];
            const BoxPar &bp = bps[box_of(nd.begin, box_off, nbox)];
            if (group_cond(nd, bp)) f = (nd.parent == kNone || !group_cond(nodes[nd.parent], bp)) ? 1u : 0u;
        }
        flag[n] = f;
    }
}

void launch_group_flags(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const uint32_t *box_off,
                        int nbox, const BoxPar *bps, uint32_t *flag, cudaStream_t s, int nsm)
{
    k_group_flags<<<nsm * 8, 256, 0, s>>>(nodes, n_nodes, node_cap, box_off, nbox, bps, flag);
    g_launches++;
}

__global__ void __launch_bounds__(256) k_group_fill(const Node *__restrict__ nodes,
                                                    const uint32_t *__restrict__ n_nodes, uint32_t node_cap,
                                                    const uint32_t *__restrict__ flag,
                                                    const uint32_t *__restrict__ gidx,
                                                    const uint32_t *__restrict__ box_off, int nbox,
                                                    Group *__restrict__ groups)
{
    const uint32_t nn = node_count(n_nodes, node_cap);
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += gridDim.x * blockDim.x) {
        if (!flag[n]) continue;
        const Node nd = nodes[n];
        const int k = nd.lvl & 255u;
        const int32_t h = 1 << (kMaxLevel - k);
        Group g;
        g.node = n;
        g.begin = nd.begin;
        g.count = nd.end - nd.begin;
        g.box = (uint32_t)box_of(nd.begin, box_off, nbox);
        g.cx = 2 * (int32_t)nd.ix + h;
        g.cy = 2 * (int32_t)nd.iy + h;
        g.cz = 2 * (int32_t)nd.iz + h;
        g.hg = h;
        groups[gidx[n]] = g;
    }
}

void launch_group_fill(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const uint32_t *flag,
                       const uint32_t *gidx, const uint32_t *box_off, int nbox, Group *groups, cudaStream_t s, int nsm)
{
    k_group_fill<<<nsm * 8, 256, 0, s>>>(nodes, n_nodes, node_cap, flag, gidx, box_off, nbox, groups);
    g_launches++;
}

// The box of finest-level cells that holds a group's particles, one warp per group:
// centre minus the group's cell centre and half sides, in u (cells lo..hi span
// [2 lo, 2 hi + 2]).  The list builder prunes against it (Eq. 2 vanishes beyond r_cut).
__global__ void __launch_bounds__(256) k_group_box(const Group *__restrict__ groups,
                                                   const uint32_t *__restrict__ n_groups,
                                                   const unsigned long long *__restrict__ pcell,
                                                   int4 *__restrict__ gbox)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t G = *n_groups;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
        const Group gr = groups[g];
        uint32_t lo[3] = {0x1fffffu, 0x1fffffu, 0x1fffffu}, hi[3] = {0u, 0u, 0u};
        for (uint32_t j = gr.begin + lane; j < gr.begin + gr.count; j += 32) {
            const unsigned long long c = pcell[j];
            const uint32_t q[3] = {(uint32_t)c & 0x1fffffu, (uint32_t)(c >> 21) & 0x1fffffu, (uint32_t)(c >> 42)};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                lo[a] = min(lo[a], q[a]);
                hi[a] = max(hi[a], q[a]);
            }
        }
        int b[3], h[3];
        const int gc[3] = {gr.cx, gr.cy, gr.cz};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int l = (int)__reduce_min_sync(FULL, lo[a]);
            const int u = (int)__reduce_max_sync(FULL, hi[a]);
            b[a] = l + u + 1 - gc[a];
            h[a] = u - l + 1;
        }
        if (lane == 0) {
            gbox[2 * (size_t)g] = make_int4(b[0], b[1], b[2], 0);
            gbox[2 * (size_t)g + 1] = make_int4(h[0], h[1], h[2], 0);
        }
    }
}

void launch_group_box(const Group *groups, const uint32_t *n_groups, const unsigned long long *pcell, int4 *gbox,
                      cudaStream_t s, int nsm)
{
    k_group_box<<<nsm * 8, 256, 0, s>>>(groups, n_groups, pcell, gbox);
    g_launches++;
}

__global__ void k_record_counts(const uint32_t *n_nodes, const uint32_t *n_groups, DevStatus *st, uint32_t node_cap)
{
    st->n_nodes = *n_nodes;
    st->n_groups = n_groups ? *n_groups : 0;
    if (*n_nodes > node_cap) atomicOr(&st->flags, ST_NODE_CAP);
}

void launch_record_counts(const uint32_t *n_nodes, const uint32_t *n_groups, DevStatus *st, uint32_t node_cap,
                          cudaStream_t s)
{
    k_record_counts<<<1, 1, 0, s>>>(n_nodes, n_groups, st, node_cap);
    g_launches++;
}

}  // namespace greem
