// Internal definitions shared by the CUDA translation units of libgreem.so.
// Nothing here is visible through the C ABI (include/greem.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace greem {

constexpr int kMaxLevel = 21;           // 21 bits per axis in a 63-bit Morton key (Sec. 3.2.5)
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kHalfPeriod = 1 << 21;    // L/2 in units u = L/2^22
constexpr int kPeriod = 1 << 22;        // L in units u

// Four doubles, 32-byte aligned (node moments: x, y, z, mass).
struct __align__(32) Dbl4 {
    double x, y, z, w;
};
__host__ __device__ __forceinline__ Dbl4 make_dbl4(double x, double y, double z, double w)
{
    Dbl4 r;
    r.x = x; r.y = y; r.z = z; r.w = w;
    return r;
}

// One tree node, 32 bytes, nodes stored in DFS preorder (a node's subtree is the
// contiguous index range [n, skip)).
struct __align__(16) Node {
    uint32_t ix, iy, iz;   // lower corner of the cell in finest-level cells (L/2^21)
    uint32_t lvl;          // level in bits 0-7, leaf flag in bit 8
    uint32_t begin, end;   // sorted particle range
    uint32_t skip;         // first node after this subtree
    uint32_t parent;       // kNone for the root of a box
};
static_assert(sizeof(Node) == 32, "Node must be 32 bytes");

// One interaction-list group (a node of at most n_crit particles, Sec. 3.1.2).
struct __align__(16) Group {
    uint32_t node, begin, count, box;
    int32_t cx, cy, cz;    // cell centre in units u = L/2^22
    int32_t hg;            // half side in u
};
static_assert(sizeof(Group) == 32, "Group must be 32 bytes");

// Per-box constants, derived on the host from greem_params.
struct BoxPar {
    // The FP32 path works in units of r_cut (offsets, list entries, i-particles); the FP64
    // form and Eq. 12 work in units of eta = r_cut/2.
    double L, inv_L, u, eta, inv_eta, inv_rc, eps;
    float k_f;             // u/r_cut rounded to float: cell offsets -> r_cut units
    float k52_f;           // (L/2^52)/r_cut rounded to float: fixed52 offsets -> r_cut units
    float inv_rc2;         // 1/r_cut^2: r_cut-unit accelerations -> physical
    float eps2;            // (eps/r_cut)^2
    long long T_prune;     // prune a node iff S_gap > T_prune (exact form of the r_cut test)
    long long A[22];       // accept a node of level k iff S_d > A[k] (exact form of the theta test)
    uint32_t p_begin, p_end;
    int lmin, n_crit, n_leaf, soft;
    int pow2_e;            // L = 2^pow2_e exactly, or kNotPow2
    // The list walk's start level K (0: every walk starts at the root) and its table of
    // level-K cells (8^K entries at tbl_off in ListArgs::tbl); rprune > sqrt(T_prune).
    int kstart, rprune;
    unsigned long long tbl_off;
};
constexpr int kNotPow2 = -100000;

// Polls of a bounded device wait before it gives up and records ST_TIMEOUT.
constexpr uint32_t kWaitPolls = 1u << 22;

// Launch state that the runtime keeps per device (a kernel's shared-memory opt-in, an
// occupancy query) is cached per device index below this bound; devices beyond it are
// not cached (the attribute is set and the occupancy queried on every launch).
constexpr int kMaxDevices = 64;
int current_device_index();  // the current device, or -1 when it is not cached

// Device status word and counters, cleared at the start of every call.
struct DevStatus {
    unsigned int flags;
    unsigned int pad;
    unsigned long long n_nodes;
    unsigned long long n_groups;
    unsigned long long list_pages;     // pages requested from the list pool
    unsigned long long sum_len;        // sum of unpadded list lengths
    unsigned long long sum_inter;      // sum of n_g * unpadded list length
    unsigned long long sum_eval;       // pair evaluations of the force kernel
    unsigned long long sum_padded;     // sum of padded list lengths (the pool demand)
    unsigned long long work[4];        // persistent-kernel work queues
    unsigned long long sum_quad;       // entries the quadrupole lists need (on overflow)
    unsigned long long sum_start;      // list walks started from a start table
    unsigned long long sum_coarse;     // leaves above the start level taken from a table
};

enum : unsigned {
    ST_NONFINITE = 1u,
    ST_NODE_CAP = 2u,
    ST_LIST_CAP = 4u,
    ST_TIMEOUT = 8u,
    ST_STACK = 16u,
    ST_QLIST_CAP = 32u,
};

// Launch shape of the list builder (warps per block, blocks per SM): every warp may
// hold one partly used page of the list pool.
#ifndef GREEM_LIST_BLOCKS
#define GREEM_LIST_BLOCKS 4
#endif
constexpr int kListWarps = 8;
constexpr int kListBlocksPerSM = GREEM_LIST_BLOCKS;

// Kernel launches made by the current host thread (reported in greem_stats).
extern thread_local long long g_launches;

// x in [0, L) with L = 2^e: floor(x 2^(52-e)), i.e. x in units of L/2^52, read from the
// bits of x with integer operations (exact for x >= L/2, truncated below 2^-52 L for
// smaller x).  Cell centres are exact in these units, so an offset from a centre is one
// integer subtraction.
__device__ __forceinline__ long long fixed52(double x, int e)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;
    const unsigned long long mant = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = (ex - 1023) - e;  // x 2^(52-e) = mant 2^sh
    if (sh >= 0) return sh > 10 ? (1ll << 62) : (long long)(mant << sh);
    return -sh >= 64 ? 0 : (long long)(mant >> (-sh));
}

// Periodic wrap into [0, L): r = x - L floor(x/L); r < 0 -> r + L; r >= L -> r - L;
// anything still outside [0, L) -> 0.  Each FP64 step is rounded separately (no FMA).
__device__ __forceinline__ double wrap_pos(double x, double L)
{
    // x in [0, L) already: floor(x/L) = 0 and the formula returns x unchanged
    if (x >= 0.0 && x < L) return x;
    double f = floor(__ddiv_rn(x, L));
    double r = __dsub_rn(x, __dmul_rn(L, f));
    if (r < 0.0) r = __dadd_rn(r, L);
    if (r >= L) r = __dsub_rn(r, L);
    if (!(r >= 0.0 && r < L)) r = 0.0;
    return r;
}

// The FP64 formula as a real call: inlined, the compiler may predicate it, and every
// lane then issues its FP64 instructions (64 cycles per warp instruction on this GPU).
static __device__ __noinline__ double wrap_pos_call(double x, double L) { return wrap_pos(x, L); }

// Wrap with the in-range test done on the bit pattern (non-negative doubles order like
// their bits): x in [0, L) returns x unchanged; anything else takes the FP64 formula.
__device__ __forceinline__ double wrap_pos_fast(double x, double L)
{
    const long long bx = __double_as_longlong(x), bl = __double_as_longlong(L);
    if (bx >= 0 && bx < bl) return x;
    return wrap_pos_call(x, L);
}

// Box of sorted/input particle i: box_off holds nbox+1 increasing offsets.
__device__ __forceinline__ int box_of(uint32_t i, const uint32_t *__restrict__ box_off, int nbox)
{
    int lo = 0, hi = nbox;  // box_off[lo] <= i < box_off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (box_off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- host launchers
struct ScanScratch {
    uint32_t *buf = nullptr;  // block sums for every level
    size_t cap = 0;
};
size_t scan_scratch_elems(size_t n);
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.  in may alias out.
void scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *scratch, cudaStream_t s);

// S1-S2 (keys_sort.cu)
void launch_keys(const double *pos, uint32_t N, const uint32_t *box_off, int nbox, const BoxPar *bps,
                 uint64_t *keys, DevStatus *st, cudaStream_t s);
size_t radix_hist_elems(uint32_t n);
size_t radix_status_elems(uint32_t n);
size_t radix_runs_elems(uint32_t n);
int radix_key_passes();
void radix_sort(uint64_t *k0, uint64_t *k1, uint32_t *v0, uint32_t *v1, uint32_t n, int key_passes, int box_passes,
                const uint32_t *box_off, int nbox, uint32_t *hist, unsigned long long *status, uint32_t *runs,
                DevStatus *st, uint64_t **k_out, uint32_t **v_out, cudaStream_t s, int nsm);
void launch_gather(const double *pos, const float *mass, const uint32_t *perm, uint32_t N, const uint32_t *box_off,
                   int nbox, const BoxPar *bps, double *xs, double *ys, double *zs, float *ms, DevStatus *st,
                   cudaStream_t s);

// S3-S4 (tree.cu)
void launch_tree_prep(const uint64_t *keys, uint32_t N, const uint32_t *box_off, int nbox, const BoxPar *bps,
                      uint8_t *d8, uint8_t *K8, uint32_t *own, cudaStream_t s);
void launch_tree_fill(const uint64_t *keys, uint32_t N, const uint32_t *box_off, int nbox, const uint8_t *d8,
                      const uint8_t *K8, const uint32_t *base, Node *nodes, uint32_t node_cap, DevStatus *st,
                      cudaStream_t s, int nsm);
void launch_tree_links(Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, uint8_t *nchild, uint32_t *kids,
                       cudaStream_t s, int nsm);
void launch_moments(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const uint32_t *kids,
                    const uint32_t *base, uint32_t N, const double *xs, const double *ys, const double *zs,
                    const float *ms, Dbl4 *raw, uint32_t *lvl, uint32_t *inodes, cudaStream_t s, int nsm);
void launch_quadrupoles(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const uint32_t *kids,
                        const float4 *poff, const float4 *noff, const uint32_t *lvl, const uint32_t *inodes,
                        const uint32_t *box_off, int nbox, const BoxPar *bps, float4 *quad, cudaStream_t s, int nsm);
void launch_leaf_boxes(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap,
                       const unsigned long long *pcell, unsigned long long *lbox, cudaStream_t s, int nsm);
void launch_leaf_offsets(const uint64_t *keys, const uint8_t *K8, uint32_t N, const uint32_t *box_off, int nbox,
                         const BoxPar *bps, const double *xs, const double *ys, const double *zs, const float *ms,
                         float4 *poff, unsigned long long *pcell, cudaStream_t s);
void launch_node_finish(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const Dbl4 *raw,
                        const uint32_t *box_off, int nbox, const BoxPar *bps, Dbl4 *mom64, float4 *noff,
                        cudaStream_t s, int nsm);
void launch_group_flags(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const uint32_t *box_off,
                        int nbox, const BoxPar *bps, uint32_t *flag, cudaStream_t s, int nsm);
void launch_group_fill(const Node *nodes, const uint32_t *n_nodes, uint32_t node_cap, const uint32_t *flag,
                       const uint32_t *gidx, const uint32_t *box_off, int nbox, Group *groups, cudaStream_t s,
                       int nsm);
void launch_group_box(const Group *groups, const uint32_t *n_groups, const unsigned long long *pcell, int4 *gbox,
                      cudaStream_t s, int nsm);
void launch_record_counts(const uint32_t *n_nodes, const uint32_t *n_groups, DevStatus *st, uint32_t node_cap,
                          cudaStream_t s);

// S5 (lists.cu)
struct ListArgs {
    const Node *nodes;
    const Group *groups;
    const uint32_t *n_groups;
    const uint32_t *base;      // node index of the first node starting at each particle (N+1)
    const BoxPar *bps;
    const uint32_t *kids;      // child table, 8 slots per node (kNone = unused)
    uint32_t *stack;           // per-warp traversal stacks
    uint32_t stack_cap;        // entries per warp stack
    const float4 *poff;        // per sorted particle: offset from its leaf centre (r_cut units), mass
    const float4 *noff;        // per node: COM offset from its cell centre (r_cut units), mass
    const unsigned long long *pcell;  // per sorted particle: finest cell, x | y << 21 | z << 42
    const unsigned long long *lbox;   // per leaf: its particles' box of finest cells (k_leaf_boxes)
    const int4 *gbox;          // per group: particle box centre minus cell centre, then half sides (u)
    float4 *flist;             // list pool, FP32 relative entries
    unsigned long long *ilist; // list pool, index entries (may be null)
    float4 *irel;              // per sorted particle: its own relative position in its group's frame
    unsigned long long *loff;  // per group: first entry
    uint32_t *llen;            // per group: padded length (multiple of 8)
    uint32_t *lraw;            // per group: unpadded length
    uint32_t *qcnt;            // per group: accepted node entries (may be null)
    unsigned long long cap;    // entries in the pool
    uint32_t page;             // entries per page
    const uint32_t *tbl;       // start tables of the boxes with kstart > 0 (k_start_table)
    DevStatus *st;
};
void launch_lists(const ListArgs &a, cudaStream_t s, int nsm);
// The start tables: for every box with kstart = K > 0, the node of each level-K cell
// (Morton order), the leaf above it with bit 31 set, or kNone where the cell is empty.
// kmax: the largest kstart over the boxes.
void launch_start_table(const Node *nodes, const uint32_t *kids, const uint32_t *base, const BoxPar *bps, int nbox,
                        int kmax, uint32_t *tbl, const DevStatus *st, cudaStream_t s);

// S6 (force.cu)
struct ForceArgs {
    const Group *groups;
    const uint32_t *n_groups;
    const uint32_t *order;     // work order over groups (may be null = identity)
    const unsigned long long *loff;
    const uint32_t *llen;
    const uint32_t *lraw;
    const float4 *flist;
    const unsigned long long *ilist;
    const float4 *irel;
    const uint32_t *perm;
    const BoxPar *bps;
    // quadrupole passes: per group the first entry and count in qlist (three float4 each)
    const uint32_t *qoff;
    const uint32_t *qcnt;
    const float4 *qlist;
    // FP64 form
    const double *xs, *ys, *zs;
    const float *ms;
    const Dbl4 *mom64;
    void *acc;
    DevStatus *st;
    int chunk;                 // list entries per staged chunk
    int warps;                 // warps per block
    // polls of each list-chunk wait, plus one (0: kWaitPolls); only a failure test
    // lowers it, through greem_debug_set
    uint32_t wait_polls1 = 0;
};
void launch_force_order(const Group *groups, const uint32_t *n_groups, uint32_t *bins, uint32_t *order,
                        cudaStream_t s, int nsm);
// Dynamic shared memory of the FP32 force kernel, and its limit: the 227 KB a block may
// opt in to, less room for the kernel's static shared memory (its mbarriers).
size_t force_smem_bytes(int chunk, int warps);
constexpr size_t kForceSmemMax = 226 * 1024;
void launch_force_f32(const ForceArgs &a, cudaStream_t s, int nsm, bool soft, bool quad = false);
void launch_qlist_fill(const ForceArgs &a, const float4 *quad, unsigned long long qcap, cudaStream_t s, int nsm);
void launch_force_f64(const ForceArgs &a, cudaStream_t s, int nsm);
void launch_pair_setup(const double *xg, const double *xi, const double *xj, const float *mj, uint32_t np,
                       double inv_rc, Group *groups, float4 *irel, float4 *flist, unsigned long long *loff,
                       uint32_t *llen, uint32_t *lraw, uint32_t *perm, uint32_t *n_groups, cudaStream_t s);
double peak_tflops(int which, int nsm, cudaStream_t s, int *err);

// Domains and local essential trees (domain.cu)
struct LetBox {
    long long c[3];  // centre of a domain box, units u = L/2^22
    long long h[3];  // half sides, units u
};
constexpr int kMaxDomains = 1024;
constexpr int kLetChunk = 16;  // receiving boxes handled by one set of LET passes
void launch_cells(const double *pos, uint32_t npos, const int64_t *idx, uint32_t n, double L, int pow2_e,
                  int32_t *cells, DevStatus *st, cudaStream_t s);
size_t dom_count_smem(int ndom);
size_t dom_scatter_smem(int ndom);
uint32_t dom_blocks(uint32_t N);
void launch_dom_count(const double *pos, uint32_t N, double L, int pow2_e, const int32_t *boxes, int ndom,
                      uint32_t *dom, uint32_t *cnt, DevStatus *st, cudaStream_t s);
void launch_dom_scatter(const double *pos, const float *mass, const int64_t *ids, uint32_t N, double L,
                        const uint32_t *dom, const uint32_t *off, int ndom, double *pos_out, float *mass_out,
                        int64_t *ids_out, cudaStream_t s);
void launch_let_count(const Node *nodes, const uint32_t *n_nodes, uint32_t ncap, const LetBox *b, int nb,
                      const BoxPar *bps, const unsigned long long *pcell, uint32_t *flag, uint32_t *cnt, cudaStream_t s,
                      int nsm);
void launch_let_ends(const uint32_t *off, uint32_t ncap, int nb, uint32_t *ends, cudaStream_t s);
void launch_let_fill(const Node *nodes, const uint32_t *n_nodes, uint32_t ncap, const LetBox *b, int nb,
                     const BoxPar *bps, const unsigned long long *pcell, const uint32_t *flag, const uint32_t *off,
                     const double *xs, const double *ys, const double *zs, const float *ms, const Dbl4 *mom64,
                     double *pos_out, float *mass_out, int64_t *ref_out, unsigned long long base, cudaStream_t s,
                     int nsm);

// PM (pm.cu)
void launch_pm_table(int n, double L, double r_cut, int scheme, float *table, cudaStream_t s, int nsm);

// time integration (integrate.cu)
void launch_kick(float *vel, const float *acc, uint32_t N, float f, cudaStream_t s, int nsm);
void launch_drift(double *pos, const float *vel, uint32_t N, double f, double L, cudaStream_t s, int nsm);
void launch_vmax_amax(const float *vel, const float *acc, uint32_t N, unsigned int *out, cudaStream_t s, int nsm);
double timestep_eq7(double eps, double zeta, float v2max, float a2max);
double softening_eq6(double eps_fin, double z_crit, double z);
double cosmo_integral(double a0, double a1, double om, double ol, double h0, int p);

}  // namespace greem
