// Context, workspace, pipeline orchestration and the C ABI of include/greem.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cufft.h>

#include "common.cuh"
#include "greem.h"

#include "pm.cuh"

namespace greem {
thread_local long long g_launches = 0;

int current_device_index()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return dev >= 0 && dev < kMaxDevices ? dev : -1;
}
}

using namespace greem;

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
};

struct greem_ctx {
    int device = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;  // private stream for graph capture on the legacy stream
    // second stream of a call: the particle offsets and the groups run on it beside the
    // moments (fork and join by events, so the whole call stays capturable)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // S1-S2
    DBuf<uint64_t> k0, k1;
    DBuf<uint32_t> v0, v1, hist, scratch;
    DBuf<unsigned long long> rs_status;
    DBuf<uint32_t> rs_runs;
    DBuf<double> xs, ys, zs;
    DBuf<float> ms;
    // S3-S4
    DBuf<uint8_t> d8, K8, nchild;
    DBuf<uint32_t> own, base, ctr, gflag, gidx;
    DBuf<Node> nodes;
    DBuf<Dbl4> raw, mom64;
    DBuf<float4> noff, poff, irel;
    DBuf<Group> groups;
    DBuf<float4> quad, qlist;
    DBuf<uint32_t> qcnt, qoff;
    size_t qcap = 0;  // quadrupole-list entries
    DBuf<unsigned long long> pcell, lbox;
    DBuf<int4> gbox;
    // S5-S6
    DBuf<float4> flist;
    DBuf<unsigned long long> ilist, loff;
    DBuf<uint32_t> llen, lraw, kids, stack, order, bins, lvl;
    DBuf<uint32_t> tbl;   // the list walk's start tables (k_start_table)
    int tbl_kmax = 0;     // the deepest start level of the current call's boxes
    int start_cap = 7;    // the deepest level a list walk may start at (greem_debug_set)
    // per call
    DBuf<BoxPar> bps;
    DBuf<uint32_t> box_off, small;
    DBuf<DevStatus> st;
    DevStatus *st_host = nullptr;
    DevStatus *st_host_dev = nullptr;  // the device's address of st_host (mapped), or null
    BoxPar *bps_host = nullptr;
    uint32_t *box_off_host = nullptr;
    int host_boxes_cap = 0;

    // capacities
    size_t node_cap = 0;
    size_t list_cap = 0;
    uint32_t page = 0;
    uint32_t stack_cap = 4096;
    // failure tests (greem_debug_set): starting capacities of the next call (0 = the
    // usual first guess), attempts per call, and the force kernel's wait limit
    size_t next_node_cap = 0, next_list_cap = 0;
    uint32_t next_stack_cap = 0;
    int max_attempts = 6;
    uint32_t wait_polls1 = 0;

    // results of the last call
    uint64_t *ks = nullptr;
    uint32_t *perm = nullptr;
    uint32_t last_N = 0;
    int last_nbox = 0;
    bool have_tree = false, have_lists = false, have_index = false, have_quad = false;
    greem_stats stats;

    // PM
    PmPlan pm;
    DBuf<float> pm_grid, pm_table;
    DBuf<cufftComplex> pm_spec, pm_tmp;
    int pm_tab_n = 0, pm_tab_scheme = -1;
    double pm_tab_L = 0, pm_tab_rc = 0;

    // host-buffer calls: two device staging slots for inputs and results, and the copy
    // streams that fill and drain them beside the computation
    DBuf<double> hs_pos[2];
    DBuf<float> hs_mass[2];
    DBuf<unsigned char> hs_acc[2];
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};

    // domains and local essential trees
    DBuf<int32_t> dom_boxes;
    DBuf<uint32_t> dom, dom_cnt;
    DBuf<uint32_t> let_flag, let_cnt, let_ends;

    // graph
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    bool capturing = false;

    // greem_short_force_ex replays a graph of a call that repeats the previous one
    // (greem_short_force_ex below); ag_gen changes whenever a buffer is reallocated or a
    // debug setting changes, so a graph never outlives the state it was captured from
    struct CallKey {
        const void *pos, *mass, *acc;
        int64_t N;
        greem_params p;
        uint64_t gen;
    };
    // two entries, so that calls alternating between two sets of buffers (the staging
    // slots of greem_short_force_host) replay too
    static constexpr int kAgEntries = 2;
    cudaGraphExec_t ag_exec[kAgEntries] = {};
    CallKey ag_key[kAgEntries] = {}, ag_seen[kAgEntries] = {};
    long long ag_launches[kAgEntries] = {};
    bool ag_seen_valid[kAgEntries] = {};
    int ag_next = 0;  // the entry the next capture replaces
    bool ag_enabled = true;
    cudaEvent_t stage_ev[7] = {};
    uint64_t ag_gen = 0;
};

static bool cuda_ok(cudaError_t e)
{
    if (e == cudaSuccess) return true;
    cudaGetLastError();
    return false;
}

// Forgets the replayable graph of greem_short_force_ex and the call it was kept for.
static void drop_auto_graph(greem_ctx *c)
{
    for (int e = 0; e < greem_ctx::kAgEntries; e++) {
        if (c->ag_exec[e]) cudaGraphExecDestroy(c->ag_exec[e]);
        c->ag_exec[e] = nullptr;
        c->ag_seen_valid[e] = false;
    }
    c->ag_gen++;
}

template <class T>
static int ensure(greem_ctx *c, DBuf<T> &b, size_t n)
{
    if (b.n >= n && b.p) return GREEM_OK;
    if (c->capturing) return GREEM_ERR_CAPACITY;
    cudaStreamSynchronize(c->stream);
    if (c->exec) {  // a captured graph points at the old buffer: drop it
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    drop_auto_graph(c);
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    size_t nn = n + n / 8 + 64;
    if (!cuda_ok(cudaMalloc((void **)&b.p, nn * sizeof(T)))) {
        b.p = nullptr;
        return GREEM_ERR_OOM;
    }
    b.n = nn;
    return GREEM_OK;
}

template <class T>
static void release(DBuf<T> &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
}

// ------------------------------------------------------------------ parameters
// Largest integer S >= 0 with fl(fl(S) * coef) <= bound (coef > 0); the products are
// monotone in S, so "S > result" is exactly "(double)S * coef > bound".
static long long max_s_le(double coef, double bound)
{
    const double SMAX = 4.0e15;
    if (bound < 0.0) return -1;
    double est = std::floor(bound / coef);
    if (!(est < SMAX)) return (long long)SMAX;
    long long S = (long long)est;
    if (S < 0) S = 0;
    while (S > 0 && (double)S * coef > bound) S--;
    while ((double)(S + 1) * coef <= bound) S++;
    if ((double)S * coef > bound) return -1;
    return S;
}

// Eq. 2 on the host, both branches as printed (only the opening-angle thresholds use it).
static double host_g_p3m(double R)
{
    if (R < 0.0) R = -R;
    const double R2 = R * R, R3 = R2 * R, R4 = R3 * R, R5 = R4 * R, R6 = R5 * R, R7 = R6 * R, R8 = R7 * R;
    if (R < 1.0) return 1.0 - (224.0 * R3 - 224.0 * R5 + 70.0 * R6 + 48.0 * R7 - 21.0 * R8) / 140.0;
    if (R < 2.0)
        return 1.0 - (12.0 - 224.0 * R2 + 896.0 * R3 - 840.0 * R4 + 224.0 * R5 + 70.0 * R6 - 48.0 * R7 + 7.0 * R8) /
                         140.0;
    return 0.0;
}

// The accept test of Eq. 12 (Sec. 4.1) for a node of side l (u) at squared distance S
// (u^2): (double)(l*l) < theta(d)^2 * (double)S, theta(d)^2 = min(theta_max^2,
// theta0^2 / (R g(R))), R = sqrt(S) u / eta, theta_max^2 where R g(R) = 0.
static bool eq12_accept(long long l, long long S, double t02, double tmax2, double u_over_eta)
{
    const double R = std::sqrt((double)S) * u_over_eta;
    const double rg = R * host_g_p3m(R);
    double t2 = tmax2;
    if (rg > 0.0) {
        const double q = t02 / rg;
        if (q < t2) t2 = q;
    }
    return (double)(l * l) < t2 * (double)S;
}

// Largest S for which a node of side l is NOT accepted under Eq. 12.  theta(d) d grows
// with d (R / g(R) and d both increase), so the test is false below a threshold and true
// above it, and a bisection over the integers finds it; LLONG_MAX if never accepted.
static long long eq12_threshold(long long l, double t02, double tmax2, double u_over_eta)
{
    long long lo = 0, hi = 1LL << 46;  // beyond any squared distance in a box (3 * 2^42)
    if (!eq12_accept(l, hi, t02, tmax2, u_over_eta)) return LLONG_MAX;
    while (hi - lo > 1) {  // invariant: accept(lo) false (S = 0 never accepts), accept(hi) true
        const long long mid = lo + (hi - lo) / 2;
        if (eq12_accept(l, mid, t02, tmax2, u_over_eta)) hi = mid;
        else lo = mid;
    }
    return lo;
}

static int derive_box(const greem_params &p, uint32_t pb, uint32_t pe, BoxPar &bp, bool eq12)
{
    if (!(p.L > 0) || !std::isfinite(p.L)) return GREEM_ERR_INVALID_ARG;
    if (!(p.r_cut > 0) || !(p.r_cut < 0.5 * p.L)) return GREEM_ERR_INVALID_ARG;
    if (!(p.theta >= 0) || !std::isfinite(p.theta)) return GREEM_ERR_INVALID_ARG;
    if (!(p.eps >= 0) || !std::isfinite(p.eps)) return GREEM_ERR_INVALID_ARG;
    if (p.n_crit < 1 || p.n_leaf < 1) return GREEM_ERR_INVALID_ARG;
    // l_min: the shallowest level whose cell side is below L/2 - r_cut
    const double lim = 0.5 * p.L - p.r_cut;
    int lmin = -1;
    double side = p.L;
    for (int k = 0; k <= kMaxLevel; k++) {
        if (side < lim) {
            lmin = k;
            break;
        }
        side *= 0.5;
    }
    if (lmin < 0) return GREEM_ERR_INVALID_ARG;
    memset(&bp, 0, sizeof(bp));
    bp.L = p.L;
    bp.inv_L = 1.0 / p.L;
    {
        int e = 0;
        const double mfrac = std::frexp(p.L, &e);  // L = mfrac * 2^e, mfrac in [0.5, 1)
        bp.pow2_e = (mfrac == 0.5 && e - 1 > -900 && e - 1 < 900) ? e - 1 : kNotPow2;
    }
    bp.u = p.L / 4194304.0;
    bp.eta = 0.5 * p.r_cut;
    bp.inv_eta = 1.0 / bp.eta;
    bp.eps = p.eps;
    bp.inv_rc = 1.0 / p.r_cut;
    bp.k_f = (float)(bp.u / p.r_cut);
    bp.k52_f = (float)(std::ldexp(p.L, -52) / p.r_cut);
    bp.inv_rc2 = (float)(bp.inv_rc * bp.inv_rc);
    bp.eps2 = (float)((p.eps / p.r_cut) * (p.eps / p.r_cut));
    bp.soft = p.eps > 0 ? 1 : 0;
    // r_cut pruning: prune iff (double)S_gap * (u*u) > r_cut*r_cut
    bp.T_prune = max_s_le(bp.u * bp.u, p.r_cut * p.r_cut);
    // opening: accept iff (double)(l*l) < (theta*theta) * (double)S_d, l = 2^(22-k) u;
    // with Eq. 12 theta(d) replaces theta (p.theta is then its upper limit)
    const double th2 = p.theta * p.theta;
    if (eq12 && !(p.theta0 > 0 && std::isfinite(p.theta0))) return GREEM_ERR_INVALID_ARG;
    for (int k = 0; k <= kMaxLevel; k++) {
        const long long l = 1LL << (22 - k);
        if (th2 <= 0) bp.A[k] = LLONG_MAX;
        else if (eq12) bp.A[k] = eq12_threshold(l, p.theta0 * p.theta0, th2, bp.u / bp.eta);
        else bp.A[k] = max_s_le(th2, (double)(l * l));
    }
    bp.p_begin = pb;
    bp.p_end = pe;
    bp.rprune = (int)std::ceil(std::sqrt((double)bp.T_prune)) + 1;
    bp.lmin = lmin;
    bp.n_crit = p.n_crit;
    bp.n_leaf = p.n_leaf;
    return GREEM_OK;
}

// The level K at which a box's list walks start (the conditions are in lists.cu's
// header): the first level at which a node can be accepted, at most cap, and no deeper
// than the first level with at least one cell per 8 particles; 0 (walks start at the
// root) for boxes of at most 4096 particles or if K would be below 2.  A level k admits no
// accepted node when (sqrt(T_prune) + sqrt(3) h_k)^2 <= A[k], h_k the half side in u; the
// test below keeps a margin above that bound.
static int start_level(const BoxPar &bp, uint32_t n, int cap)
{
    if (cap < 2 || n <= (uint32_t)std::max(4096, bp.n_leaf)) return 0;
    int kn = 2;
    while (kn < cap && std::ldexp(1.0, 3 * kn) < n / 8.0) kn++;
    const double R = std::sqrt((double)bp.T_prune);
    for (int k = std::max(bp.lmin, 1); k < kn; k++) {
        const double v = R + 1.7320508075688772 * std::ldexp(1.0, kMaxLevel - k);
        if (v * v * (1.0 + 1e-9) + 16.0 > (double)bp.A[k]) return k >= 2 ? k : 0;
    }
    return kn;
}

static int check_common(const greem_params &p)
{
    if (p.precision != GREEM_F32_REL && p.precision != GREEM_F64) return GREEM_ERR_INVALID_ARG;
    if (p.list_chunk != 0 && (p.list_chunk < 64 || p.list_chunk > 2048 || (p.list_chunk & (p.list_chunk - 1))))
        return GREEM_ERR_INVALID_ARG;
    if (p.block_shape < 0 || p.block_shape > 16) return GREEM_ERR_INVALID_ARG;
    // the force kernel's chunk buffers must fit in one block's shared memory
    if (force_smem_bytes(p.list_chunk ? p.list_chunk : 256, p.block_shape ? p.block_shape : 16) > kForceSmemMax)
        return GREEM_ERR_INVALID_ARG;
    if ((p.flags & GREEM_FLAG_QUADRUPOLE) && (p.precision != GREEM_F32_REL || p.eps != 0.0))
        return GREEM_ERR_INVALID_ARG;
    if (p.flags & GREEM_FLAG_ADD_PM) {
        if (p.precision != GREEM_F32_REL || p.n_pm < 8 || p.n_pm > 1024) return GREEM_ERR_INVALID_ARG;
        if (p.assign != GREEM_ASSIGN_CIC && p.assign != GREEM_ASSIGN_TSC) return GREEM_ERR_INVALID_ARG;
    }
    return GREEM_OK;
}

// ------------------------------------------------------------------ PM buffers
static int pm_prepare(greem_ctx *c, int n, double L, double r_cut, int scheme)
{
    int rc;
    const size_t cells = (size_t)n * n * n, half = (size_t)n * n * (n / 2 + 1), h = (size_t)(n / 2 + 1);
    if ((rc = ensure(c, c->pm_grid, cells)) || (rc = ensure(c, c->pm_spec, half)) ||
        (rc = ensure(c, c->pm_tmp, half)) || (rc = ensure(c, c->pm_table, h * h * h)))
        return rc;
    if (!(c->pm.have && c->pm.n == n)) {
        if (c->capturing) return GREEM_ERR_CAPACITY;
        if (pm_plan(c->pm, n, c->stream)) return GREEM_ERR_CUDA;
    } else {
        pm_plan(c->pm, n, c->stream);
    }
    if (c->pm_tab_n != n || c->pm_tab_L != L || c->pm_tab_rc != r_cut || c->pm_tab_scheme != scheme) {
        if (c->capturing) return GREEM_ERR_CAPACITY;
        launch_pm_table(n, L, r_cut, scheme, c->pm_table.p, c->stream, c->nsm);
        c->pm_tab_n = n;
        c->pm_tab_L = L;
        c->pm_tab_rc = r_cut;
        c->pm_tab_scheme = scheme;
    }
    return GREEM_OK;
}

static int pow2_exponent(double L)
{
    int e = 0;
    const double mfrac = std::frexp(L, &e);
    return (mfrac == 0.5 && e - 1 > -900 && e - 1 < 900) ? e - 1 : kNotPow2;
}

// ------------------------------------------------------------------ pipeline
struct RunCfg {
    const double *pos;
    const float *mass;
    void *acc;
    uint32_t N;
    int nbox;
    int precision;
    bool index_lists;
    bool lists_force;
    bool soft;
    bool timing;
    int chunk;
    int warps;
    bool add_pm;
    int n_pm;
    int assign;
    bool quad;
};

static int host_boxes(greem_ctx *c, int nbox)
{
    if (c->host_boxes_cap >= nbox) return GREEM_OK;
    if (c->bps_host) cudaFreeHost(c->bps_host);
    if (c->box_off_host) cudaFreeHost(c->box_off_host);
    c->bps_host = nullptr;
    c->box_off_host = nullptr;
    c->host_boxes_cap = 0;
    if (!cuda_ok(cudaMallocHost((void **)&c->bps_host, sizeof(BoxPar) * nbox))) return GREEM_ERR_OOM;
    if (!cuda_ok(cudaMallocHost((void **)&c->box_off_host, sizeof(uint32_t) * (nbox + 1)))) return GREEM_ERR_OOM;
    c->host_boxes_cap = nbox;
    return GREEM_OK;
}

static uint32_t choose_page(uint32_t N, int nsm)
{
    const double warps = (double)nsm * 4 * 8;
    double per = (double)N * 32.0 / warps;
    uint32_t pg = 2048;
    while (pg < per && pg < 65536) pg <<= 1;
    return pg;
}

static int size_buffers(greem_ctx *c, const RunCfg &r)
{
    const size_t N = r.N;
    int rc;
#define ENS(b, n)                                 \
    do {                                          \
        if ((rc = ensure(c, c->b, (n))) != 0) return rc; \
    } while (0)
    ENS(k0, N);
    ENS(k1, N);
    ENS(v0, N);
    ENS(v1, N);
    ENS(hist, radix_hist_elems((uint32_t)N));
    ENS(rs_status, radix_status_elems((uint32_t)N));
    ENS(rs_runs, radix_runs_elems((uint32_t)N));
    const size_t big = std::max<size_t>(N + 1, c->node_cap + 1);
    ENS(scratch, scan_scratch_elems(big) + 64);
    ENS(xs, N);
    ENS(ys, N);
    ENS(zs, N);
    ENS(ms, N);
    ENS(d8, N);
    ENS(K8, N);
    ENS(own, N);
    ENS(base, N + 1);
    ENS(poff, N);
    ENS(pcell, N);
    ENS(irel, N);
    const size_t nc = c->node_cap;
    ENS(nodes, nc);
    ENS(nchild, nc);
    ENS(ctr, nc);
    ENS(raw, nc);
    ENS(mom64, nc);
    ENS(noff, nc);
    ENS(lbox, nc);
    ENS(gflag, nc);
    ENS(gidx, nc + 1);
    ENS(groups, nc);
    ENS(gbox, nc * 2);
    if (r.quad) {
        ENS(quad, nc * 2);
        ENS(qcnt, nc);
        ENS(qoff, nc + 1);
        ENS(qlist, c->qcap * 3);
    }
    ENS(kids, nc * 8);
    ENS(lvl, 192);
    ENS(bps, (size_t)r.nbox);
    ENS(box_off, (size_t)r.nbox + 1);
    ENS(st, 1);
    ENS(small, 16);
    if (r.lists_force) {
        ENS(loff, nc);
        ENS(llen, nc);
        ENS(lraw, nc);
        ENS(order, nc);
        ENS(bins, 128);
        ENS(stack, (size_t)c->nsm * kListBlocksPerSM * kListWarps * c->stack_cap);
        ENS(flist, c->list_cap);
        if (r.index_lists) ENS(ilist, c->list_cap);
    }
    // start levels and table offsets (multiples of 64 entries: 16-byte aligned stores);
    // a table entry flags a leaf in bit 31, so node indices must stay below 2^31
    size_t tbl_n = 0;
    c->tbl_kmax = 0;
    const bool tables = r.lists_force && nc < 0x80000000ull;
    for (int b = 0; b < r.nbox; b++) {
        BoxPar &bp = c->bps_host[b];
        const uint32_t nb = c->box_off_host[b + 1] - c->box_off_host[b];
        bp.kstart = tables ? start_level(bp, nb, c->start_cap) : 0;
        bp.tbl_off = tbl_n;
        if (bp.kstart) tbl_n += (size_t)1 << (3 * bp.kstart);
        c->tbl_kmax = std::max(c->tbl_kmax, bp.kstart);
    }
    if (tbl_n) ENS(tbl, tbl_n);
#undef ENS
    return GREEM_OK;
}

// The per-call constants of up to kInlineBoxes boxes go to the device as a kernel
// argument and the status word comes back through mapped host memory, so that a call
// issues no copy of its own: a copy would queue on the copy engines behind the
// multi-hundred-megabyte transfers that greem_short_force_host overlaps with the call.
constexpr int kInlineBoxes = 4;
static_assert(sizeof(DevStatus) % 4 == 0, "DevStatus is copied as 32-bit words");
struct InlineBoxes {
    BoxPar b[kInlineBoxes];
    uint32_t off[kInlineBoxes + 1];
    int nbox;
};

// Also clears the status word (a memset could sit on a copy engine too).
__global__ void k_set_boxes(InlineBoxes ib, BoxPar *__restrict__ bps, uint32_t *__restrict__ box_off,
                            DevStatus *__restrict__ st)
{
    const int t = threadIdx.x;
    if (t < ib.nbox) bps[t] = ib.b[t];
    if (t <= ib.nbox) box_off[t] = ib.off[t];
    uint32_t *w = reinterpret_cast<uint32_t *>(st);
    for (int i = t; i < (int)(sizeof(DevStatus) / 4); i += blockDim.x) w[i] = 0u;
}

__global__ void k_status_out(const DevStatus *__restrict__ src, DevStatus *dst)
{
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    volatile uint32_t *d = reinterpret_cast<volatile uint32_t *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(DevStatus) / 4); i += blockDim.x) d[i] = s[i];
}

// Clears the status word and uploads the per-box constants.
static void upload_boxes(greem_ctx *c, int nbox, cudaStream_t s)
{
    if (nbox <= kInlineBoxes) {
        InlineBoxes ib;
        memset(&ib, 0, sizeof(ib));
        ib.nbox = nbox;
        for (int b = 0; b < nbox; b++) ib.b[b] = c->bps_host[b];
        for (int b = 0; b <= nbox; b++) ib.off[b] = c->box_off_host[b];
        k_set_boxes<<<1, 32, 0, s>>>(ib, c->bps.p, c->box_off.p, c->st.p);
        greem::g_launches++;
    } else {
        cudaMemsetAsync(c->st.p, 0, sizeof(DevStatus), s);
        cudaMemcpyAsync(c->bps.p, c->bps_host, sizeof(BoxPar) * nbox, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(c->box_off.p, c->box_off_host, sizeof(uint32_t) * (nbox + 1), cudaMemcpyHostToDevice, s);
    }
}

static void download_status(greem_ctx *c, cudaStream_t s)
{
    if (c->st_host_dev) {
        k_status_out<<<1, 32, 0, s>>>(c->st.p, c->st_host_dev);
        greem::g_launches++;
    } else {
        cudaMemcpyAsync(c->st_host, c->st.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
    }
}

static void ev_record(greem_ctx *c, const RunCfg &r, cudaEvent_t *ev, int i)
{
    if (!r.timing || !ev) return;
    // under capture a plain record only marks a dependency; an external record becomes a
    // node of the graph that records the event each time the graph runs
    if (c->capturing) cudaEventRecordWithFlags(ev[i], c->stream, cudaEventRecordExternal);
    else cudaEventRecord(ev[i], c->stream);
}

// The stage-time events of the context (created on first use; kept, so that a captured
// call records them too), or null if they cannot be created.
static cudaEvent_t *stage_events(greem_ctx *c)
{
    if (!c->stage_ev[0])
        for (auto &e : c->stage_ev)
            if (!cuda_ok(cudaEventCreate(&e))) {
                for (auto &f : c->stage_ev)
                    if (f) cudaEventDestroy(f);
                for (auto &f : c->stage_ev) f = nullptr;
                return nullptr;
            }
    return c->stage_ev;
}

static int enqueue(greem_ctx *c, const RunCfg &r, cudaEvent_t *ev)
{
    int rc = size_buffers(c, r);
    if (rc) return rc;
    cudaStream_t s = c->stream;
    const uint32_t N = r.N;
    const int nbox = r.nbox;
    const int nsm = c->nsm;
    const uint32_t ncap = (uint32_t)std::min<size_t>(c->node_cap, 0xFFFFFFF0u);
    upload_boxes(c, nbox, s);
    ev_record(c, r, ev, 0);
    launch_keys(r.pos, N, c->box_off.p, nbox, c->bps.p, c->k0.p, c->st.p, s);
    ev_record(c, r, ev, 1);
    const int box_passes = nbox <= 1 ? 0 : (nbox <= 256 ? 1 : 2);
    uint64_t *ks = nullptr;
    uint32_t *perm = nullptr;
    radix_sort(c->k0.p, c->k1.p, c->v0.p, c->v1.p, N, radix_key_passes(), box_passes, c->box_off.p, nbox, c->hist.p,
               c->rs_status.p, c->rs_runs.p, c->st.p, &ks, &perm, s, nsm);
    launch_gather(r.pos, r.mass, perm, N, c->box_off.p, nbox, c->bps.p, c->xs.p, c->ys.p, c->zs.p, c->ms.p, c->st.p,
                  s);
    ev_record(c, r, ev, 2);
    launch_tree_prep(ks, N, c->box_off.p, nbox, c->bps.p, c->d8.p, c->K8.p, c->own.p, s);
    scan_u32(c->own.p, c->base.p, N, c->scratch.p, s);
    const uint32_t *n_nodes = c->base.p + N;
    launch_tree_fill(ks, N, c->box_off.p, nbox, c->d8.p, c->K8.p, c->base.p, c->nodes.p, ncap, c->st.p, s, nsm);
    launch_tree_links(c->nodes.p, n_nodes, ncap, c->nchild.p, c->kids.p, s, nsm);
    // fork: the moments (FP64-bound) on s; the particle offsets and the groups (integer
    // work, reading only the tree) on the second stream
    cudaStream_t s2 = c->aux;
    cudaEventRecord(c->ev_fork, s);
    cudaStreamWaitEvent(s2, c->ev_fork, 0);
    launch_leaf_offsets(ks, c->K8.p, N, c->box_off.p, nbox, c->bps.p, c->xs.p, c->ys.p, c->zs.p, c->ms.p, c->poff.p,
                        c->pcell.p, s2);
    launch_group_flags(c->nodes.p, n_nodes, ncap, c->box_off.p, nbox, c->bps.p, c->gflag.p, s2, nsm);
    scan_u32(c->gflag.p, c->gidx.p, ncap, c->scratch.p, s2);
    const uint32_t *n_groups = c->gidx.p + ncap;
    launch_group_fill(c->nodes.p, n_nodes, ncap, c->gflag.p, c->gidx.p, c->box_off.p, nbox, c->groups.p, s2, nsm);
    launch_group_box(c->groups.p, n_groups, c->pcell.p, c->gbox.p, s2, nsm);
    launch_leaf_boxes(c->nodes.p, n_nodes, ncap, c->pcell.p, c->lbox.p, s2, nsm);
    launch_record_counts(n_nodes, n_groups, c->st.p, ncap, s2);
    if (r.lists_force)
        launch_start_table(c->nodes.p, c->kids.p, c->base.p, c->bps.p, nbox, c->tbl_kmax, c->tbl.p, c->st.p, s2);
    cudaEventRecord(c->ev_join, s2);
    launch_moments(c->nodes.p, n_nodes, ncap, c->kids.p, c->base.p, N, c->xs.p, c->ys.p, c->zs.p, c->ms.p, c->raw.p,
                   c->lvl.p,
                   c->ctr.p, s, nsm);
    launch_node_finish(c->nodes.p, n_nodes, ncap, c->raw.p, c->box_off.p, nbox, c->bps.p, c->mom64.p, c->noff.p, s,
                       nsm);
    ev_record(c, r, ev, 3);
    // join: what the second stream still had to do counts as the groups stage
    cudaStreamWaitEvent(s, c->ev_join, 0);
    if (r.quad)
        launch_quadrupoles(c->nodes.p, n_nodes, ncap, c->kids.p, c->poff.p, c->noff.p, c->lvl.p, c->ctr.p,
                           c->box_off.p, nbox, c->bps.p, c->quad.p, s, nsm);
    ev_record(c, r, ev, 4);
    if (r.lists_force) {
        ListArgs la;
        la.nodes = c->nodes.p;
        la.groups = c->groups.p;
        la.n_groups = n_groups;
        la.base = c->base.p;
        la.bps = c->bps.p;
        la.kids = c->kids.p;
        la.stack = c->stack.p;
        la.stack_cap = c->stack_cap;
        la.poff = c->poff.p;
        la.noff = c->noff.p;
        la.pcell = c->pcell.p;
        la.lbox = c->lbox.p;
        la.gbox = c->gbox.p;
        la.flist = c->flist.p;
        la.ilist = r.index_lists ? c->ilist.p : nullptr;
        la.irel = c->irel.p;
        la.loff = c->loff.p;
        la.llen = c->llen.p;
        la.lraw = c->lraw.p;
        la.qcnt = r.quad ? c->qcnt.p : nullptr;
        if (r.quad) cudaMemsetAsync(c->qcnt.p, 0, sizeof(uint32_t) * ncap, s);
        la.cap = c->list_cap;
        la.page = c->page;
        la.tbl = c->tbl.p;
        la.st = c->st.p;
        launch_lists(la, s, nsm);
        ev_record(c, r, ev, 5);
        launch_force_order(c->groups.p, n_groups, c->bins.p, c->order.p, s, nsm);
        ForceArgs fa = {};
        fa.wait_polls1 = c->wait_polls1;
        fa.groups = c->groups.p;
        fa.n_groups = n_groups;
        fa.order = c->order.p;
        fa.loff = c->loff.p;
        fa.llen = c->llen.p;
        fa.lraw = c->lraw.p;
        fa.flist = c->flist.p;
        fa.ilist = r.index_lists ? c->ilist.p : nullptr;
        fa.irel = c->irel.p;
        fa.perm = perm;
        fa.bps = c->bps.p;
        fa.xs = c->xs.p;
        fa.ys = c->ys.p;
        fa.zs = c->zs.p;
        fa.ms = c->ms.p;
        fa.mom64 = c->mom64.p;
        fa.acc = r.acc;
        fa.st = c->st.p;
        fa.chunk = r.chunk;
        fa.warps = r.warps;
        if (r.precision == GREEM_F64) launch_force_f64(fa, s, nsm);
        else launch_force_f32(fa, s, nsm, r.soft);
        if (r.quad) {
            scan_u32(c->qcnt.p, c->qoff.p, ncap, c->scratch.p, s);
            fa.qoff = c->qoff.p;
            fa.qcnt = c->qcnt.p;
            fa.qlist = c->qlist.p;
            launch_qlist_fill(fa, c->quad.p, c->qcap, s, nsm);
            launch_force_f32(fa, s, nsm, false, true);
        }
        if (r.add_pm) {
            const BoxPar &b0 = c->bps_host[0];
            if ((rc = pm_prepare(c, r.n_pm, b0.L, 2.0 * b0.eta, r.assign))) return rc;
            // input order: Morton-sorted particles of dense halos make consecutive lanes hit the
            // same cells and serialise the assignment atomics
            if (run_pm(c->pm, r.pos, nullptr, nullptr, nullptr, r.mass, nullptr, N, b0.L, r.n_pm, r.assign, b0.pow2_e,
                       c->pm_table.p, c->pm_grid.p, c->pm_spec.p, c->pm_tmp.p, (float *)r.acc, 1, s, nsm))
                return GREEM_ERR_CUDA;
        }
        ev_record(c, r, ev, 6);
    }
    download_status(c, s);
    c->ks = ks;
    c->perm = perm;
    if (!cuda_ok(cudaGetLastError())) return GREEM_ERR_CUDA;
    return GREEM_OK;
}

// Waits for the stream and turns the device status into a return code.
static int finish(greem_ctx *c, const RunCfg &r, cudaEvent_t *ev)
{
    if (!cuda_ok(cudaStreamSynchronize(c->stream))) return GREEM_ERR_CUDA;
    const DevStatus &h = *c->st_host;
    greem_stats &S = c->stats;
    S.n_particles = r.N;
    S.n_boxes = r.nbox;
    S.n_nodes = (int64_t)h.n_nodes;
    S.n_groups = (int64_t)h.n_groups;
    S.n_list_entries = (int64_t)h.sum_len;
    S.n_interactions = (int64_t)h.sum_inter;
    S.n_evaluated = (int64_t)h.sum_eval;
    S.n_start_table = (int64_t)h.sum_start;
    S.n_start_coarse = (int64_t)h.sum_coarse;
    S.list_capacity = (int64_t)c->list_cap;
    S.l_min = c->bps_host[0].lmin;
    if (r.timing && ev) {
        float t[7] = {0, 0, 0, 0, 0, 0, 0};
        const int last = r.lists_force ? 6 : 4;
        for (int i = 1; i <= last; i++) cudaEventElapsedTime(&t[i], ev[i - 1], ev[i]);
        S.ms_keys = t[1];
        S.ms_sort = t[2];
        S.ms_tree = t[3];
        S.ms_groups = t[4];
        S.ms_lists = r.lists_force ? t[5] : 0;
        S.ms_force = r.lists_force ? t[6] : 0;
        float tot = 0;
        cudaEventElapsedTime(&tot, ev[0], ev[last]);
        S.ms_total = tot;
    }
    c->last_N = r.N;
    c->last_nbox = r.nbox;
    if (h.flags & ST_NONFINITE) return GREEM_ERR_INVALID_ARG;
    if (h.flags & ST_TIMEOUT) return GREEM_ERR_TIMEOUT;
    if (h.flags & (ST_NODE_CAP | ST_LIST_CAP | ST_STACK | ST_QLIST_CAP)) return GREEM_ERR_CAPACITY;
    c->have_tree = true;
    c->have_lists = r.lists_force;
    c->have_index = r.lists_force && r.index_lists;
    c->have_quad = r.quad;
    return GREEM_OK;
}

static void grow_caps(greem_ctx *c)
{
    const DevStatus &h = *c->st_host;
    if (h.flags & ST_NODE_CAP) c->node_cap = (size_t)(h.n_nodes * 1.15) + 4096;
    if (h.flags & ST_QLIST_CAP) c->qcap = std::max<size_t>(c->qcap * 2, (size_t)(h.sum_quad * 1.25) + 4096);
    if (h.flags & ST_STACK) c->stack_cap *= 4;
    if (h.flags & ST_LIST_CAP) {
        // every allocation abandons less than the list that did not fit, and every warp
        // holds at most one partly used page
        const size_t warps = (size_t)c->nsm * kListBlocksPerSM * kListWarps;
        const size_t need = (size_t)(2.0 * (double)h.sum_padded) + warps * c->page;
        c->list_cap = std::max<size_t>(c->list_cap + c->list_cap / 2, need);
    }
}

static int run(greem_ctx *c, RunCfg r)
{
    c->have_tree = c->have_lists = c->have_index = c->have_quad = false;
    // first guesses; an overflow grows them and the call is retried
    if (c->next_node_cap) c->node_cap = c->next_node_cap;
    else if (c->node_cap < (size_t)(r.N * 0.5) + 4096u * r.nbox) c->node_cap = (size_t)(r.N * 0.75) + 4096u * r.nbox;
    if (c->next_stack_cap) c->stack_cap = c->next_stack_cap;
    uint32_t pg = choose_page(r.N, c->nsm);
    if (pg > c->page) c->page = pg;
    if (r.lists_force) {
        const size_t warps = (size_t)c->nsm * kListBlocksPerSM * kListWarps;
        if (c->next_list_cap) c->list_cap = c->next_list_cap;
        else c->list_cap = std::max<size_t>(c->list_cap, (size_t)r.N * 32 + warps * c->page);
        // accepted nodes are a minority of the entries: a first guess of 4 per particle
        if (r.quad) c->qcap = std::max<size_t>(c->qcap, (size_t)r.N * 4 + 4096);
    }
    c->next_node_cap = c->next_list_cap = 0;
    c->next_stack_cap = 0;
    cudaEvent_t *ev = r.timing ? stage_events(c) : nullptr;
    int rc = GREEM_OK;
    c->stats.retries = 0;
    c->stats.replayed = 0;
    for (int attempt = 0; attempt < c->max_attempts; attempt++) {
        greem::g_launches = 0;
        rc = enqueue(c, r, ev);
        if (rc == GREEM_OK) rc = finish(c, r, ev);
        c->stats.kernel_launches = greem::g_launches;
        if (rc != GREEM_ERR_CAPACITY) break;
        grow_caps(c);
        c->stats.retries++;
    }
    return rc;
}

static int setup_single(greem_ctx *c, int64_t N, const greem_params *p)
{
    if (!c || !p || N < 1 || N >= (int64_t)0x7FFFFFF0) return GREEM_ERR_INVALID_ARG;
    int rc = check_common(*p);
    if (rc) return rc;
    if ((rc = host_boxes(c, 1))) return rc;
    if ((rc = derive_box(*p, 0, (uint32_t)N, c->bps_host[0], (p->flags & GREEM_FLAG_THETA_EQ12) != 0))) return rc;
    c->box_off_host[0] = 0;
    c->box_off_host[1] = (uint32_t)N;
    return GREEM_OK;
}

static RunCfg make_cfg(const greem_params &p, const double *pos, const float *mass, void *acc, uint32_t N, int nbox,
                       bool lists_force)
{
    RunCfg r;
    r.pos = pos;
    r.mass = mass;
    r.acc = acc;
    r.N = N;
    r.nbox = nbox;
    r.precision = p.precision;
    r.quad = (p.flags & GREEM_FLAG_QUADRUPOLE) != 0;
    r.index_lists = (p.flags & GREEM_FLAG_INDEX_LISTS) || p.precision == GREEM_F64 || r.quad;
    r.lists_force = lists_force;
    r.soft = false;
    r.timing = (p.flags & GREEM_FLAG_STAGE_TIMES) != 0;
    r.chunk = p.list_chunk ? p.list_chunk : 256;
    r.warps = p.block_shape ? p.block_shape : 16;
    r.add_pm = (p.flags & GREEM_FLAG_ADD_PM) != 0;
    r.n_pm = p.n_pm;
    r.assign = p.assign;
    return r;
}

// Device staging for the host-buffer calls: grown before any copy is in flight, and
// never part of a captured graph.
template <class T>
static int ensure_staging(DBuf<T> &b, size_t n)
{
    if (b.n >= n && b.p) return GREEM_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    if (!cuda_ok(cudaMalloc((void **)&b.p, n * sizeof(T)))) {
        b.p = nullptr;
        return GREEM_ERR_OOM;
    }
    b.n = n;
    return GREEM_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

void greem_params_default(greem_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->L = 1.0;
    p->r_cut = 3.0 / 32.0;
    p->theta = 0.5;
    p->eps = 0.0;
    p->n_crit = 64;
    p->n_leaf = 10;
    p->precision = GREEM_F32_REL;
    p->theta0 = 0.25;
}

int greem_create(greem_ctx **out, void *cuda_stream)
{
    if (!out) return GREEM_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev))) return GREEM_ERR_CUDA;
    cudaDeviceProp prop;
    if (!cuda_ok(cudaGetDeviceProperties(&prop, dev))) return GREEM_ERR_CUDA;
    greem_ctx *c = new (std::nothrow) greem_ctx();
    if (!c) return GREEM_ERR_OOM;
    c->device = dev;
    c->nsm = prop.multiProcessorCount;
    c->stream = (cudaStream_t)cuda_stream;
    memset(&c->stats, 0, sizeof(c->stats));
    if (!cuda_ok(cudaMallocHost((void **)&c->st_host, sizeof(DevStatus)))) {
        delete c;
        return GREEM_ERR_OOM;
    }
    memset(c->st_host, 0, sizeof(DevStatus));
    {
        void *dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, c->st_host, 0) == cudaSuccess) c->st_host_dev = static_cast<DevStatus *>(dp);
        else cudaGetLastError();  // not mapped: the status comes back by a copy
    }
    if (!cuda_ok(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking)) ||
        !cuda_ok(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) ||
        !cuda_ok(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming))) {
        greem_destroy(c);
        return GREEM_ERR_CUDA;
    }
    *out = c;
    return GREEM_OK;
}

void greem_destroy(greem_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    for (auto &g : c->ag_exec)
        if (g) cudaGraphExecDestroy(g);
    for (auto &e : c->stage_ev)
        if (e) cudaEventDestroy(e);
    pm_plan_destroy(c->pm);
    release(c->pm_grid); release(c->pm_table); release(c->pm_spec); release(c->pm_tmp);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    for (cudaStream_t hs : {c->h2d, c->d2h})
        if (hs) {
            cudaStreamSynchronize(hs);
            cudaStreamDestroy(hs);
        }
    for (int k = 0; k < 2; k++) {
        if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
        if (c->ev_out[k]) cudaEventDestroy(c->ev_out[k]);
        release(c->hs_pos[k]); release(c->hs_mass[k]); release(c->hs_acc[k]);
    }
    if (c->aux) cudaStreamSynchronize(c->aux);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    release(c->k0); release(c->k1); release(c->v0); release(c->v1); release(c->hist); release(c->scratch);
    release(c->rs_status); release(c->rs_runs);
    release(c->xs); release(c->ys); release(c->zs); release(c->ms);
    release(c->d8); release(c->K8); release(c->nchild); release(c->own); release(c->base); release(c->ctr);
    release(c->gflag); release(c->gidx); release(c->nodes); release(c->raw); release(c->mom64); release(c->noff);
    release(c->poff); release(c->pcell); release(c->lbox); release(c->irel); release(c->groups); release(c->gbox); release(c->quad);
    release(c->flist); release(c->ilist); release(c->loff);
    release(c->llen); release(c->lraw); release(c->kids); release(c->stack); release(c->order); release(c->bins);
    release(c->lvl); release(c->bps); release(c->box_off); release(c->small); release(c->st);
    release(c->qlist); release(c->qcnt); release(c->qoff);
    release(c->dom_boxes); release(c->dom); release(c->dom_cnt); release(c->let_flag); release(c->let_cnt);
    release(c->let_ends); release(c->tbl);
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->bps_host) cudaFreeHost(c->bps_host);
    if (c->box_off_host) cudaFreeHost(c->box_off_host);
    delete c;
}

int greem_build_tree(greem_ctx *c, const double *pos, const float *mass, int64_t N, const greem_params *p)
{
    int rc = setup_single(c, N, p);
    if (rc) return rc;
    if (!pos || !mass) return GREEM_ERR_INVALID_ARG;
    return run(c, make_cfg(*p, pos, mass, nullptr, (uint32_t)N, 1, false));
}

// Captures the whole call (the kernels of enqueue, both streams) into c->ag_exec[slot],
// on the context's own stream (the legacy stream cannot be captured); the graph is
// launched on the context's stream.  Nothing runs during the capture.  A capture that
// fails leaves no graph and turns the context's replays off; the calls run as usual.
static void capture_auto_graph(greem_ctx *c, const RunCfg &r, const greem_ctx::CallKey &key, int slot)
{
    if (!c->own_stream && !cuda_ok(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking))) return;
    cudaStream_t user = c->stream;
    c->stream = c->own_stream;
    c->capturing = true;
    const long long launches = greem::g_launches;
    greem::g_launches = 0;
    cudaGraph_t g = nullptr;
    int rc = GREEM_ERR_CUDA;
    if (cuda_ok(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal))) {
        rc = enqueue(c, r, r.timing ? stage_events(c) : nullptr);
        if (!cuda_ok(cudaStreamEndCapture(c->stream, &g))) rc = GREEM_ERR_CUDA;
    }
    c->capturing = false;
    c->stream = user;
    c->ag_launches[slot] = greem::g_launches;
    greem::g_launches = launches;
    if (rc == GREEM_OK && g && cuda_ok(cudaGraphInstantiate(&c->ag_exec[slot], g, 0))) {
        c->ag_key[slot] = key;
    } else {
        c->ag_exec[slot] = nullptr;
        c->ag_enabled = false;  // not retried on every later call
    }
    if (g) cudaGraphDestroy(g);
}

// A call that repeats one of the two previous ones (the same device pointers, N,
// parameters, buffers and debug settings) replays a graph of it: the whole step in one
// launch, with the same kernels and results (stage times included: the context's stage
// events are recorded by the graph).  The graph is captured after the second such call;
// if a capture fails, the context stops replaying.  A replay whose new positions
// overflow a capacity falls back to the usual call, which grows the buffers (and drops
// the graph) and retries.  Calls with the PM part never replay.
int greem_short_force_ex(greem_ctx *c, const double *pos, const float *mass, int64_t N, const greem_params *p,
                         void *acc)
{
    int rc = setup_single(c, N, p);
    if (rc) return rc;
    if (!pos || !mass || !acc) return GREEM_ERR_INVALID_ARG;
    RunCfg r = make_cfg(*p, pos, mass, acc, (uint32_t)N, 1, true);
    r.soft = p->eps > 0;
    const bool eligible = c->ag_enabled && !r.add_pm && !c->capturing;
    greem_ctx::CallKey key;
    auto make_key = [&]() {
        memset(&key, 0, sizeof(key));
        key.pos = pos;
        key.mass = mass;
        key.acc = acc;
        key.N = N;
        key.p = *p;
        key.gen = c->ag_gen;
    };
    auto same = [](const greem_ctx::CallKey &a, const greem_ctx::CallKey &b) { return !memcmp(&a, &b, sizeof(a)); };
    c->stats.replayed = 0;
    constexpr int E = greem_ctx::kAgEntries;
    if (eligible) {
        make_key();
        for (int e = 0; e < E; e++) {
            if (!c->ag_exec[e] || !same(key, c->ag_key[e])) continue;
            c->have_tree = c->have_lists = c->have_index = c->have_quad = false;
            if (!cuda_ok(cudaGraphLaunch(c->ag_exec[e], c->stream))) return GREEM_ERR_CUDA;
            rc = finish(c, r, r.timing ? stage_events(c) : nullptr);
            c->stats.kernel_launches = c->ag_launches[e];
            c->stats.retries = 0;
            if (rc != GREEM_ERR_CAPACITY) {
                c->stats.replayed = 1;
                return rc;
            }
            grow_caps(c);  // the usual call below reallocates, which drops the graphs
            break;
        }
    }
    rc = run(c, r);
    if (rc == GREEM_OK && eligible) {
        make_key();  // run() may have reallocated: the generation is the current one
        int seen = -1;
        for (int e = 0; e < E; e++)
            if (c->ag_seen_valid[e] && same(key, c->ag_seen[e])) seen = e;
        if (seen >= 0) {
            // the second call of this kind among the recent ones: capture it for the next
            int slot = -1;
            for (int e = 0; e < E; e++)
                if (c->ag_exec[e] && same(key, c->ag_key[e])) slot = e;
            if (slot < 0) {
                slot = c->ag_next;
                c->ag_next = (c->ag_next + 1) % E;
                if (c->ag_exec[slot]) cudaGraphExecDestroy(c->ag_exec[slot]);
                c->ag_exec[slot] = nullptr;
                capture_auto_graph(c, r, key, slot);
            }
        } else {
            // remember it in place of the older of the recent calls
            for (int e = E - 1; e > 0; e--) {
                c->ag_seen[e] = c->ag_seen[e - 1];
                c->ag_seen_valid[e] = c->ag_seen_valid[e - 1];
            }
            c->ag_seen[0] = key;
            c->ag_seen_valid[0] = true;
        }
    }
    return rc;
}

int greem_short_force_host(greem_ctx *c, int nstep, const double *const *pos, const float *const *mass,
                           const int64_t *N, const greem_params *p, void *const *acc)
{
    if (!c || !p || nstep < 1 || !pos || !mass || !N || !acc || c->capturing) return GREEM_ERR_INVALID_ARG;
    int64_t nmax = 0;
    for (int k = 0; k < nstep; k++) {
        if (!pos[k] || !mass[k] || !acc[k] || N[k] < 1 || N[k] >= (int64_t)0x7FFFFFF0) return GREEM_ERR_INVALID_ARG;
        nmax = std::max(nmax, N[k]);
    }
    const size_t esz = p->precision == GREEM_F64 ? sizeof(double) : sizeof(float);
    if (!c->h2d) {
        if (!cuda_ok(cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking)) ||
            !cuda_ok(cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking)))
            return GREEM_ERR_CUDA;
        for (int k = 0; k < 2; k++)
            if (!cuda_ok(cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming)) ||
                !cuda_ok(cudaEventCreateWithFlags(&c->ev_out[k], cudaEventDisableTiming)))
                return GREEM_ERR_CUDA;
    }
    // nothing may be in flight on the copy streams while the slots are resized
    if (!cuda_ok(cudaStreamSynchronize(c->h2d)) || !cuda_ok(cudaStreamSynchronize(c->d2h))) return GREEM_ERR_CUDA;
    int rc = GREEM_OK;
    for (int k = 0; k < 2 && rc == GREEM_OK; k++)
        (rc = ensure_staging(c->hs_pos[k], 3 * (size_t)nmax)) || (rc = ensure_staging(c->hs_mass[k], (size_t)nmax)) ||
            (rc = ensure_staging(c->hs_acc[k], 3 * (size_t)nmax * esz));
    if (rc) return rc;
    // inputs of problem k into slot k & 1, on the copy-in stream
    auto copy_in = [&](int k) {
        const int s = k & 1;
        const bool ok =
            cuda_ok(cudaMemcpyAsync(c->hs_pos[s].p, pos[k], 3 * sizeof(double) * (size_t)N[k], cudaMemcpyHostToDevice,
                                    c->h2d)) &&
            cuda_ok(cudaMemcpyAsync(c->hs_mass[s].p, mass[k], sizeof(float) * (size_t)N[k], cudaMemcpyHostToDevice,
                                    c->h2d)) &&
            cuda_ok(cudaEventRecord(c->ev_in[s], c->h2d));
        return ok;
    };
    if (!copy_in(0)) rc = GREEM_ERR_CUDA;
    for (int k = 0; k < nstep && rc == GREEM_OK; k++) {
        const int s = k & 1;
        // the other slot's inputs were last read by problem k-1, which has finished
        if (k + 1 < nstep && !copy_in(k + 1)) {
            rc = GREEM_ERR_CUDA;
            break;
        }
        // problem k starts when its inputs have landed and the result that last used this
        // slot (problem k-2) has been copied out
        if (!cuda_ok(cudaStreamWaitEvent(c->stream, c->ev_in[s], 0)) ||
            (k >= 2 && !cuda_ok(cudaStreamWaitEvent(c->stream, c->ev_out[s], 0)))) {
            rc = GREEM_ERR_CUDA;
            break;
        }
        rc = greem_short_force_ex(c, c->hs_pos[s].p, c->hs_mass[s].p, N[k], p, c->hs_acc[s].p);
        if (rc) break;
        // the call waited for its stream: the result is complete; copy it out beside the
        // next problem
        if (!cuda_ok(cudaMemcpyAsync(acc[k], c->hs_acc[s].p, 3 * esz * (size_t)N[k], cudaMemcpyDeviceToHost, c->d2h)) ||
            !cuda_ok(cudaEventRecord(c->ev_out[s], c->d2h)))
            rc = GREEM_ERR_CUDA;
    }
    // the slots must be idle before the call returns, also after a failure
    const bool idle = cuda_ok(cudaStreamSynchronize(c->h2d)) && cuda_ok(cudaStreamSynchronize(c->d2h));
    if (rc == GREEM_OK && !idle) rc = GREEM_ERR_CUDA;
    return rc;
}

static std::mutex g_def_mu;
static greem_ctx *g_def_ctx[256];

int greem_short_force(const double *pos, const float *mass, int64_t N, double L, double r_cut, double theta,
                      int n_crit, float *acc)
{
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev)) || dev < 0 || dev >= 256) return GREEM_ERR_CUDA;
    greem_ctx *c;
    {
        std::lock_guard<std::mutex> lk(g_def_mu);
        if (!g_def_ctx[dev]) {
            int rc = greem_create(&g_def_ctx[dev], nullptr);
            if (rc) return rc;
        }
        c = g_def_ctx[dev];
    }
    greem_params p;
    greem_params_default(&p);
    p.L = L;
    p.r_cut = r_cut;
    p.theta = theta;
    p.n_crit = n_crit;
    std::lock_guard<std::mutex> lk(g_def_mu);
    return greem_short_force_ex(c, pos, mass, N, &p, acc);
}

int greem_short_force_batched(greem_ctx *c, int nbox, const int64_t *offsets, const double *pos, const float *mass,
                              const greem_params *per_box, void *acc)
{
    if (!c || !offsets || !per_box || !pos || !mass || !acc) return GREEM_ERR_INVALID_ARG;
    if (nbox < 1 || nbox > 65536) return GREEM_ERR_INVALID_ARG;
    if (offsets[0] != 0) return GREEM_ERR_INVALID_ARG;
    for (int b = 0; b < nbox; b++)
        if (offsets[b + 1] <= offsets[b]) return GREEM_ERR_INVALID_ARG;
    const int64_t N = offsets[nbox];
    if (N >= (int64_t)0x7FFFFFF0) return GREEM_ERR_INVALID_ARG;
    int rc = check_common(per_box[0]);
    if (rc) return rc;
    if ((rc = host_boxes(c, nbox))) return rc;
    bool soft = false;
    for (int b = 0; b < nbox; b++) {
        if ((rc = derive_box(per_box[b], (uint32_t)offsets[b], (uint32_t)offsets[b + 1], c->bps_host[b],
                             (per_box[0].flags & GREEM_FLAG_THETA_EQ12) != 0)))
            return rc;
        c->box_off_host[b] = (uint32_t)offsets[b];
        soft = soft || per_box[b].eps > 0;
    }
    c->box_off_host[nbox] = (uint32_t)N;
    RunCfg r = make_cfg(per_box[0], pos, mass, acc, (uint32_t)N, nbox, true);
    r.soft = soft;
    if (r.quad && soft) return GREEM_ERR_INVALID_ARG;
    return run(c, r);
}

int greem_pm_force(greem_ctx *c, const double *pos, const float *mass, int64_t N, double L, int n_pm, double r_cut,
                   int assign, float *acc_pm)
{
    if (!c || !pos || !mass || !acc_pm || N < 1 || N >= (int64_t)0x7FFFFFF0) return GREEM_ERR_INVALID_ARG;
    if (!(L > 0) || !std::isfinite(L) || !(r_cut > 0) || !(r_cut < 0.5 * L)) return GREEM_ERR_INVALID_ARG;
    if (n_pm < 8 || n_pm > 1024 || (assign != GREEM_ASSIGN_CIC && assign != GREEM_ASSIGN_TSC))
        return GREEM_ERR_INVALID_ARG;
    int rc = pm_prepare(c, n_pm, L, r_cut, assign);
    if (rc) return rc;
    greem::g_launches = 0;
    if (run_pm(c->pm, pos, nullptr, nullptr, nullptr, mass, nullptr, (uint32_t)N, L, n_pm, assign, pow2_exponent(L),
               c->pm_table.p, c->pm_grid.p, c->pm_spec.p, c->pm_tmp.p, acc_pm, 0, c->stream, c->nsm))
        return GREEM_ERR_CUDA;
    if (!cuda_ok(cudaGetLastError()) || !cuda_ok(cudaStreamSynchronize(c->stream))) return GREEM_ERR_CUDA;
    c->stats.kernel_launches = greem::g_launches;
    return GREEM_OK;
}

int greem_graph_capture(greem_ctx *c, const double *pos, const float *mass, int64_t N, const greem_params *p, void *acc)
{
    int rc = greem_short_force_ex(c, pos, mass, N, p, acc);
    if (rc) return rc;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    cudaStream_t user = c->stream;
    if (!user) {
        if (!c->own_stream && !cuda_ok(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking)))
            return GREEM_ERR_CUDA;
        cudaStreamSynchronize(nullptr);
        c->stream = c->own_stream;
    }
    RunCfg r = make_cfg(*p, pos, mass, acc, (uint32_t)N, 1, true);
    r.soft = p->eps > 0;
    r.timing = false;
    cudaGraph_t g = nullptr;
    c->capturing = true;
    greem::g_launches = 0;
    if (!cuda_ok(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal))) {
        c->capturing = false;
        c->stream = user;
        return GREEM_ERR_CUDA;
    }
    rc = enqueue(c, r, nullptr);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->capturing = false;
    c->graph_stream = c->stream;
    c->stream = user;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (!cuda_ok(e)) return GREEM_ERR_CUDA;
    e = cudaGraphInstantiate(&c->exec, g, 0);
    cudaGraphDestroy(g);
    if (!cuda_ok(e)) {
        c->exec = nullptr;
        return GREEM_ERR_CUDA;
    }
    c->stats.kernel_launches = greem::g_launches;
    return GREEM_OK;
}

int greem_graph_launch(greem_ctx *c)
{
    if (!c || !c->exec) return GREEM_ERR_INVALID_ARG;
    if (c->graph_stream != c->stream) cudaStreamSynchronize(c->stream);
    if (!cuda_ok(cudaGraphLaunch(c->exec, c->graph_stream))) return GREEM_ERR_CUDA;
    if (!cuda_ok(cudaStreamSynchronize(c->graph_stream))) return GREEM_ERR_CUDA;
    const DevStatus &h = *c->st_host;
    c->stats.n_nodes = (int64_t)h.n_nodes;
    c->stats.n_groups = (int64_t)h.n_groups;
    c->stats.n_list_entries = (int64_t)h.sum_len;
    c->stats.n_interactions = (int64_t)h.sum_inter;
    c->stats.n_evaluated = (int64_t)h.sum_eval;
    if (h.flags & ST_NONFINITE) return GREEM_ERR_INVALID_ARG;
    if (h.flags & ST_TIMEOUT) return GREEM_ERR_TIMEOUT;
    if (h.flags & (ST_NODE_CAP | ST_LIST_CAP | ST_STACK | ST_QLIST_CAP)) return GREEM_ERR_CAPACITY;
    return GREEM_OK;
}

int greem_get_stats(greem_ctx *c, greem_stats *out)
{
    if (!c || !out) return GREEM_ERR_INVALID_ARG;
    *out = c->stats;
    return GREEM_OK;
}

int greem_debug_dump(greem_ctx *c, int what, void *host_buf, int64_t cap_bytes, int64_t *len_bytes)
{
    if (!c || !len_bytes) return GREEM_ERR_INVALID_ARG;
    *len_bytes = 0;
    if (!c->have_tree) return GREEM_ERR_INVALID_ARG;
    const uint32_t N = c->last_N;
    const uint32_t nn = (uint32_t)c->stats.n_nodes;
    const uint32_t G = (uint32_t)c->stats.n_groups;
    if (!cuda_ok(cudaStreamSynchronize(c->stream))) return GREEM_ERR_CUDA;
    switch (what) {
    case GREEM_DUMP_KEYS: {
        *len_bytes = (int64_t)N * 8;
        if (!host_buf || cap_bytes < *len_bytes) return GREEM_ERR_INVALID_ARG;
        return cuda_ok(cudaMemcpy(host_buf, c->ks, (size_t)N * 8, cudaMemcpyDeviceToHost)) ? 0 : GREEM_ERR_CUDA;
    }
    case GREEM_DUMP_PERM: {
        *len_bytes = (int64_t)N * 4;
        if (!host_buf || cap_bytes < *len_bytes) return GREEM_ERR_INVALID_ARG;
        return cuda_ok(cudaMemcpy(host_buf, c->perm, (size_t)N * 4, cudaMemcpyDeviceToHost)) ? 0 : GREEM_ERR_CUDA;
    }
    case GREEM_DUMP_NODES: {
        *len_bytes = (int64_t)nn * 9 * 8;
        if (!host_buf || cap_bytes < *len_bytes) return GREEM_ERR_INVALID_ARG;
        std::vector<Node> h(nn);
        if (!cuda_ok(cudaMemcpy(h.data(), c->nodes.p, (size_t)nn * sizeof(Node), cudaMemcpyDeviceToHost)))
            return GREEM_ERR_CUDA;
        int64_t *o = (int64_t *)host_buf;
        for (uint32_t n = 0; n < nn; n++) {
            const int k = h[n].lvl & 255u;
            o[9 * n + 0] = k;
            o[9 * n + 1] = h[n].ix >> (kMaxLevel - k);
            o[9 * n + 2] = h[n].iy >> (kMaxLevel - k);
            o[9 * n + 3] = h[n].iz >> (kMaxLevel - k);
            o[9 * n + 4] = h[n].begin;
            o[9 * n + 5] = h[n].end;
            o[9 * n + 6] = h[n].skip;
            o[9 * n + 7] = (h[n].lvl >> 8) & 1u;
            o[9 * n + 8] = h[n].parent == kNone ? -1 : (int64_t)h[n].parent;
        }
        return GREEM_OK;
    }
    case GREEM_DUMP_MOMENTS: {
        *len_bytes = (int64_t)nn * 4 * 8;
        if (!host_buf || cap_bytes < *len_bytes) return GREEM_ERR_INVALID_ARG;
        std::vector<Dbl4> h(nn);
        if (!cuda_ok(cudaMemcpy(h.data(), c->mom64.p, (size_t)nn * sizeof(Dbl4), cudaMemcpyDeviceToHost)))
            return GREEM_ERR_CUDA;
        double *o = (double *)host_buf;
        for (uint32_t n = 0; n < nn; n++) {
            o[4 * n] = h[n].w;
            o[4 * n + 1] = h[n].x;
            o[4 * n + 2] = h[n].y;
            o[4 * n + 3] = h[n].z;
        }
        return GREEM_OK;
    }
    case GREEM_DUMP_GROUPS: {
        *len_bytes = (int64_t)G * 8;
        if (!host_buf || cap_bytes < *len_bytes) return GREEM_ERR_INVALID_ARG;
        std::vector<Group> h(G);
        if (G && !cuda_ok(cudaMemcpy(h.data(), c->groups.p, (size_t)G * sizeof(Group), cudaMemcpyDeviceToHost)))
            return GREEM_ERR_CUDA;
        int64_t *o = (int64_t *)host_buf;
        for (uint32_t g = 0; g < G; g++) o[g] = h[g].node;
        return GREEM_OK;
    }
    case GREEM_DUMP_QUADRUPOLES: {
        if (!c->have_quad) return GREEM_ERR_INVALID_ARG;
        *len_bytes = (int64_t)nn * 6 * 8;
        if (!host_buf || cap_bytes < *len_bytes) return GREEM_ERR_INVALID_ARG;
        std::vector<float4> h((size_t)nn * 2);
        std::vector<Node> hn(nn);
        if (nn && (!cuda_ok(cudaMemcpy(h.data(), c->quad.p, (size_t)nn * 2 * sizeof(float4), cudaMemcpyDeviceToHost)) ||
                   !cuda_ok(cudaMemcpy(hn.data(), c->nodes.p, (size_t)nn * sizeof(Node), cudaMemcpyDeviceToHost))))
            return GREEM_ERR_CUDA;
        double *o = (double *)host_buf;
        int b = 0;
        for (uint32_t n = 0; n < nn; n++) {
            while (b + 1 < c->last_nbox && hn[n].begin >= c->box_off_host[b + 1]) b++;
            const double rc = 2.0 * c->bps_host[b].eta, e2 = rc * rc;  // r_cut^2 units -> physical
            const float4 q0 = h[2 * (size_t)n], q1 = h[2 * (size_t)n + 1];
            o[6 * n + 0] = q0.x * e2;
            o[6 * n + 1] = q0.y * e2;
            o[6 * n + 2] = q0.z * e2;
            o[6 * n + 3] = q0.w * e2;
            o[6 * n + 4] = q1.x * e2;
            o[6 * n + 5] = q1.y * e2;
        }
        return GREEM_OK;
    }
    case GREEM_DUMP_LIST_OFFSETS:
    case GREEM_DUMP_LISTS: {
        if (!c->have_lists) return GREEM_ERR_INVALID_ARG;
        std::vector<uint32_t> raw(G);
        std::vector<unsigned long long> off(G);
        if (G && (!cuda_ok(cudaMemcpy(raw.data(), c->lraw.p, (size_t)G * 4, cudaMemcpyDeviceToHost)) ||
                  !cuda_ok(cudaMemcpy(off.data(), c->loff.p, (size_t)G * 8, cudaMemcpyDeviceToHost))))
            return GREEM_ERR_CUDA;
        int64_t tot = 0;
        for (uint32_t g = 0; g < G; g++) tot += raw[g];
        if (what == GREEM_DUMP_LIST_OFFSETS) {
            *len_bytes = (int64_t)(G + 1) * 8;
            if (!host_buf || cap_bytes < *len_bytes) return GREEM_ERR_INVALID_ARG;
            int64_t *o = (int64_t *)host_buf;
            o[0] = 0;
            for (uint32_t g = 0; g < G; g++) o[g + 1] = o[g] + raw[g];
            return GREEM_OK;
        }
        if (!c->have_index) return GREEM_ERR_INVALID_ARG;
        *len_bytes = tot * 5 * 8;
        if (!host_buf || cap_bytes < *len_bytes) return GREEM_ERR_INVALID_ARG;
        size_t used = 0;
        for (uint32_t g = 0; g < G; g++) used = std::max<size_t>(used, off[g] + raw[g]);
        std::vector<unsigned long long> pool(used);
        if (used && !cuda_ok(cudaMemcpy(pool.data(), c->ilist.p, used * 8, cudaMemcpyDeviceToHost)))
            return GREEM_ERR_CUDA;
        std::vector<Node> hn(nn);
        if (nn && !cuda_ok(cudaMemcpy(hn.data(), c->nodes.p, (size_t)nn * sizeof(Node), cudaMemcpyDeviceToHost)))
            return GREEM_ERR_CUDA;
        // entries are disjoint particle ranges: sorting by first particle restores preorder
        auto first = [&](unsigned long long v) -> uint64_t {
            const uint32_t ix = (uint32_t)v;
            return ((v >> 32) & 1ull) ? hn[ix].begin : ix;
        };
        for (uint32_t g = 0; g < G; g++) {
            auto *b = pool.data() + off[g];
            std::sort(b, b + raw[g],
                      [&](unsigned long long x, unsigned long long y) { return first(x) < first(y); });
        }
        int64_t *o = (int64_t *)host_buf;
        int64_t e = 0;
        auto dec = [](unsigned v) -> int64_t { return v == 1u ? 1 : (v == 2u ? -1 : 0); };
        for (uint32_t g = 0; g < G; g++) {
            for (uint32_t t = 0; t < raw[g]; t++, e++) {
                const unsigned long long v = pool[off[g] + t];
                const unsigned code = (unsigned)(v >> 33) & 63u;
                o[5 * e + 0] = (int64_t)((v >> 32) & 1ull);
                o[5 * e + 1] = (int64_t)(uint32_t)v;
                o[5 * e + 2] = dec(code & 3u);
                o[5 * e + 3] = dec((code >> 2) & 3u);
                o[5 * e + 4] = dec((code >> 4) & 3u);
            }
        }
        return GREEM_OK;
    }
    default:
        return GREEM_ERR_INVALID_ARG;
    }
}

int greem_debug_dump_group_lists(greem_ctx *c, const int64_t *groups, int64_t ngroups, int64_t *offsets,
                                 int64_t *entries, int64_t cap_entries, int64_t *n_entries)
{
    if (!c || !groups || !offsets || !n_entries || ngroups < 0) return GREEM_ERR_INVALID_ARG;
    *n_entries = 0;
    if (!c->have_lists || !c->have_index) return GREEM_ERR_INVALID_ARG;
    const int64_t G = c->stats.n_groups;
    if (!cuda_ok(cudaStreamSynchronize(c->stream))) return GREEM_ERR_CUDA;
    for (int64_t k = 0; k < ngroups; k++)
        if (groups[k] < 0 || groups[k] >= G) return GREEM_ERR_INVALID_ARG;
    std::vector<uint32_t> raw_all((size_t)G);
    std::vector<unsigned long long> off_all((size_t)G);
    if (G && (!cuda_ok(cudaMemcpy(raw_all.data(), c->lraw.p, (size_t)G * 4, cudaMemcpyDeviceToHost)) ||
              !cuda_ok(cudaMemcpy(off_all.data(), c->loff.p, (size_t)G * 8, cudaMemcpyDeviceToHost))))
        return GREEM_ERR_CUDA;
    std::vector<uint32_t> raw(ngroups);
    std::vector<unsigned long long> off(ngroups);
    int64_t tot = 0;
    for (int64_t k = 0; k < ngroups; k++) {
        raw[k] = raw_all[(size_t)groups[k]];
        off[k] = off_all[(size_t)groups[k]];
        offsets[k] = tot;
        tot += raw[k];
    }
    offsets[ngroups] = tot;
    *n_entries = tot;
    if (!entries || cap_entries < tot) return tot ? GREEM_ERR_INVALID_ARG : GREEM_OK;
    auto dec = [](unsigned v) -> int64_t { return v == 1u ? 1 : (v == 2u ? -1 : 0); };
    // first particle of each entry (node begin for nodes) gives preorder: the nodes come
    // to the host in one copy
    const size_t nn = (size_t)c->stats.n_nodes;
    std::vector<Node> nodes(nn);
    if (nn && !cuda_ok(cudaMemcpy(nodes.data(), c->nodes.p, nn * sizeof(Node), cudaMemcpyDeviceToHost)))
        return GREEM_ERR_CUDA;
    std::vector<unsigned long long> buf;
    int64_t e = 0;
    for (int64_t k = 0; k < ngroups; k++) {
        buf.resize(raw[k]);
        if (raw[k] && !cuda_ok(cudaMemcpy(buf.data(), c->ilist.p + off[k], (size_t)raw[k] * 8, cudaMemcpyDeviceToHost)))
            return GREEM_ERR_CUDA;
        std::vector<std::pair<uint64_t, unsigned long long>> keyed(raw[k]);
        for (uint32_t t = 0; t < raw[k]; t++) {
            const unsigned long long v = buf[t];
            uint64_t first = (uint32_t)v;
            if ((v >> 32) & 1ull) {
                if ((uint32_t)v >= nn) return GREEM_ERR_INVALID_ARG;
                first = nodes[(uint32_t)v].begin;
            }
            keyed[t] = {first, v};
        }
        std::sort(keyed.begin(), keyed.end());
        for (uint32_t t = 0; t < raw[k]; t++, e++) {
            const unsigned long long v = keyed[t].second;
            const unsigned code = (unsigned)(v >> 33) & 63u;
            entries[5 * e + 0] = (int64_t)((v >> 32) & 1ull);
            entries[5 * e + 1] = (int64_t)(uint32_t)v;
            entries[5 * e + 2] = dec(code & 3u);
            entries[5 * e + 3] = dec((code >> 2) & 3u);
            entries[5 * e + 4] = dec((code >> 4) & 3u);
        }
    }
    return GREEM_OK;
}

int greem_debug_dump_group_entries(greem_ctx *c, const int64_t *groups, int64_t ngroups, int64_t *offsets,
                                   float *entries, int64_t *index_entries, int64_t cap_entries, int64_t *n_entries)
{
    if (!c || !groups || !offsets || !n_entries || ngroups < 0) return GREEM_ERR_INVALID_ARG;
    *n_entries = 0;
    if (!c->have_lists || (index_entries && !c->have_index)) return GREEM_ERR_INVALID_ARG;
    const int64_t G = c->stats.n_groups;
    if (!cuda_ok(cudaStreamSynchronize(c->stream))) return GREEM_ERR_CUDA;
    for (int64_t k = 0; k < ngroups; k++)
        if (groups[k] < 0 || groups[k] >= G) return GREEM_ERR_INVALID_ARG;
    // list lengths and offsets of every group in one copy each
    std::vector<uint32_t> raw_all((size_t)G);
    std::vector<unsigned long long> off_all((size_t)G);
    if (G && (!cuda_ok(cudaMemcpy(raw_all.data(), c->lraw.p, (size_t)G * 4, cudaMemcpyDeviceToHost)) ||
              !cuda_ok(cudaMemcpy(off_all.data(), c->loff.p, (size_t)G * 8, cudaMemcpyDeviceToHost))))
        return GREEM_ERR_CUDA;
    int64_t tot = 0;
    for (int64_t k = 0; k < ngroups; k++) {
        offsets[k] = tot;
        tot += raw_all[(size_t)groups[k]];
    }
    offsets[ngroups] = tot;
    *n_entries = tot;
    if (!entries || cap_entries < tot) return tot ? GREEM_ERR_INVALID_ARG : GREEM_OK;
    auto dec = [](unsigned v) -> int64_t { return v == 1u ? 1 : (v == 2u ? -1 : 0); };
    std::vector<unsigned long long> buf;
    for (int64_t k = 0; k < ngroups; k++) {
        const size_t g = (size_t)groups[k];
        const uint32_t n = raw_all[g];
        if (!n) continue;
        if (!cuda_ok(cudaMemcpy(entries + 4 * offsets[k], c->flist.p + off_all[g], (size_t)n * sizeof(float4),
                                cudaMemcpyDeviceToHost)))
            return GREEM_ERR_CUDA;
        if (!index_entries) continue;
        buf.resize(n);
        if (!cuda_ok(cudaMemcpy(buf.data(), c->ilist.p + off_all[g], (size_t)n * 8, cudaMemcpyDeviceToHost)))
            return GREEM_ERR_CUDA;
        for (uint32_t t = 0; t < n; t++) {
            const unsigned long long v = buf[t];
            const unsigned code = (unsigned)(v >> 33) & 63u;
            int64_t *o = index_entries + 5 * (offsets[k] + t);
            o[0] = (int64_t)((v >> 32) & 1ull);
            o[1] = (int64_t)(uint32_t)v;
            o[2] = dec(code & 3u);
            o[3] = dec((code >> 2) & 3u);
            o[4] = dec((code >> 4) & 3u);
        }
    }
    return GREEM_OK;
}

int greem_autotune(greem_ctx *c, const double *pos, const float *mass, int64_t N, const greem_params *p,
                   const int *candidates, int ncand, void *acc, greem_params *best)
{
    if (!c || !p || !best) return GREEM_ERR_INVALID_ARG;
    static const int def_cand[] = {32, 48, 64, 96, 128, 160, 192, 256, 384, 512};
    if (!candidates || ncand <= 0) {
        candidates = def_cand;
        ncand = (int)(sizeof(def_cand) / sizeof(def_cand[0]));
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timeit = [&](const greem_params &q, float *ms) -> int {
        int rc = greem_short_force_ex(c, pos, mass, N, &q, acc);  // warm (sizes buffers)
        if (rc) return rc;
        float bestms = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(e0, c->stream);
            rc = greem_short_force_ex(c, pos, mass, N, &q, acc);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            if (rc) return rc;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            bestms = std::min(bestms, t);
        }
        *ms = bestms;
        return GREEM_OK;
    };
    greem_params cur = *p;
    cur.flags &= ~GREEM_FLAG_INDEX_LISTS;
    float bt = 1e30f;
    int rc = GREEM_OK;
    greem_params bp = cur;
    auto tryq = [&](const greem_params &q) -> int {
        float t;
        const int r = timeit(q, &t);
        if (!r && t < bt) {
            bt = t;
            bp = q;
        }
        return r;
    };
    // 1. n_crit at the given shape (unset fields: the default shape)
    int ib = 0;
    for (int i = 0; i < ncand && !rc; i++) {
        greem_params q = cur;
        q.n_crit = candidates[i];
        const float before = bt;
        rc = tryq(q);
        if (bt < before) ib = i;
    }
    // 2. list chunk and block shape at that n_crit
    if (!rc) {
        const int chunks[] = {128, 256, 512, 1024};
        const int shapes[] = {4, 8, 16};
        const greem_params base = bp;
        for (int ci = 0; ci < 4 && !rc; ci++)
            for (int si = 0; si < 3 && !rc; si++) {
                greem_params q = base;
                q.list_chunk = chunks[ci];
                q.block_shape = shapes[si];
                if (force_smem_bytes(q.list_chunk, q.block_shape) > kForceSmemMax) continue;
                rc = tryq(q);
            }
    }
    // 3. the neighbouring n_crit candidates again at the chosen shape (the best n_crit
    // depends on the shape)
    if (!rc) {
        const greem_params base = bp;
        for (int i = ib - 1; i <= ib + 1 && !rc; i += 2) {
            if (i < 0 || i >= ncand) continue;
            greem_params q = base;
            q.n_crit = candidates[i];
            rc = tryq(q);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    bp.flags = p->flags;
    *best = bp;
    return GREEM_OK;
}

int greem_pair_force_f32(greem_ctx *c, const double *x_g, const double *x_i, const double *x_j, const float *m_j,
                         int64_t npairs, double r_cut, double eps, float *acc)
{
    if (!c || !x_g || !x_i || !x_j || !m_j || !acc) return GREEM_ERR_INVALID_ARG;
    if (npairs < 1 || npairs >= (int64_t)0x0FFFFFFF || !(r_cut > 0) || !(eps >= 0)) return GREEM_ERR_INVALID_ARG;
    const size_t np = (size_t)npairs;
    int rc;
    if ((rc = ensure(c, c->groups, np)) || (rc = ensure(c, c->irel, np)) || (rc = ensure(c, c->flist, 8 * np)) ||
        (rc = ensure(c, c->loff, np)) || (rc = ensure(c, c->llen, np)) || (rc = ensure(c, c->lraw, np)) ||
        (rc = ensure(c, c->v0, np)) || (rc = ensure(c, c->bps, 1)) || (rc = ensure(c, c->st, 1)) ||
        (rc = ensure(c, c->small, 16)))
        return rc;
    if ((rc = host_boxes(c, 1))) return rc;
    BoxPar &bp = c->bps_host[0];
    memset(&bp, 0, sizeof(bp));
    bp.eta = 0.5 * r_cut;
    bp.inv_eta = 1.0 / bp.eta;
    bp.inv_rc = 1.0 / r_cut;
    bp.inv_rc2 = (float)(bp.inv_rc * bp.inv_rc);
    bp.eps = eps;
    bp.eps2 = (float)((eps / r_cut) * (eps / r_cut));
    cudaStream_t s = c->stream;
    greem::g_launches = 0;
    if (!cuda_ok(cudaMemsetAsync(c->st.p, 0, sizeof(DevStatus), s)) ||
        !cuda_ok(cudaMemcpyAsync(c->bps.p, c->bps_host, sizeof(BoxPar), cudaMemcpyHostToDevice, s)))
        return GREEM_ERR_CUDA;
    launch_pair_setup(x_g, x_i, x_j, m_j, (uint32_t)np, bp.inv_rc, c->groups.p, c->irel.p, c->flist.p, c->loff.p,
                      c->llen.p, c->lraw.p, c->v0.p, c->small.p, s);
    if (!cuda_ok(cudaGetLastError())) return GREEM_ERR_CUDA;
    ForceArgs fa = {};
    fa.wait_polls1 = c->wait_polls1;
    fa.groups = c->groups.p;
    fa.n_groups = c->small.p;
    fa.order = nullptr;
    fa.loff = c->loff.p;
    fa.llen = c->llen.p;
    fa.lraw = c->lraw.p;
    fa.flist = c->flist.p;
    fa.irel = c->irel.p;
    fa.perm = c->v0.p;
    fa.bps = c->bps.p;
    fa.acc = acc;
    fa.st = c->st.p;
    fa.chunk = 256;
    fa.warps = 8;
    launch_force_f32(fa, s, c->nsm, eps > 0);
    if (!cuda_ok(cudaGetLastError())) return GREEM_ERR_CUDA;
    if (!cuda_ok(cudaMemcpyAsync(c->st_host, c->st.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, s)) ||
        !cuda_ok(cudaStreamSynchronize(s)))
        return GREEM_ERR_CUDA;
    c->have_tree = c->have_lists = c->have_index = c->have_quad = false;
    if (c->st_host->flags & ST_TIMEOUT) return GREEM_ERR_TIMEOUT;
    return GREEM_OK;
}

int greem_kick(greem_ctx *c, float *vel, const float *acc, int64_t N, double f_kick)
{
    if (!c || !vel || !acc || N < 1 || N >= (int64_t)0x7FFFFFF0 || !std::isfinite(f_kick)) return GREEM_ERR_INVALID_ARG;
    greem::g_launches = 0;
    launch_kick(vel, acc, (uint32_t)N, (float)f_kick, c->stream, c->nsm);
    if (!cuda_ok(cudaGetLastError())) return GREEM_ERR_CUDA;
    c->stats.kernel_launches = greem::g_launches;
    return GREEM_OK;
}

int greem_drift(greem_ctx *c, double *pos, const float *vel, int64_t N, double L, double f_drift)
{
    if (!c || !pos || !vel || N < 1 || N >= (int64_t)0x7FFFFFF0 || !(L > 0) || !std::isfinite(L) ||
        !std::isfinite(f_drift))
        return GREEM_ERR_INVALID_ARG;
    greem::g_launches = 0;
    launch_drift(pos, vel, (uint32_t)N, f_drift, L, c->stream, c->nsm);
    if (!cuda_ok(cudaGetLastError())) return GREEM_ERR_CUDA;
    c->stats.kernel_launches = greem::g_launches;
    return GREEM_OK;
}

int greem_timestep(greem_ctx *c, const float *vel, const float *acc, int64_t N, double eps, double zeta, double *dt)
{
    if (!c || !vel || !acc || !dt || N < 1 || N >= (int64_t)0x7FFFFFF0 || !(eps > 0) || !(zeta > 0))
        return GREEM_ERR_INVALID_ARG;
    int rc;
    if ((rc = ensure(c, c->small, 16))) return rc;
    launch_vmax_amax(vel, acc, (uint32_t)N, c->small.p, c->stream, c->nsm);
    unsigned int h[2] = {0, 0};
    if (!cuda_ok(cudaMemcpyAsync(h, c->small.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream)) ||
        !cuda_ok(cudaStreamSynchronize(c->stream)))
        return GREEM_ERR_CUDA;
    float v2, a2;
    memcpy(&v2, &h[0], 4);
    memcpy(&a2, &h[1], 4);
    *dt = timestep_eq7(eps, zeta, v2, a2);
    return GREEM_OK;
}

double greem_softening(double eps_fin, double z_crit, double z) { return softening_eq6(eps_fin, z_crit, z); }

int greem_cosmo_factors(double a0, double a1, double omega_m, double omega_l, double h0, double *kick, double *drift)
{
    if (!kick || !drift || !(a0 > 0) || !(a1 > a0) || !(h0 > 0) || !std::isfinite(a1)) return GREEM_ERR_INVALID_ARG;
    // H^2 must stay positive on [a0, a1] (checked on 65 points spanning it)
    for (int i = 0; i <= 64; i++) {
        const double a = a0 + (a1 - a0) * i / 64.0;
        if (!(omega_m / (a * a * a) + (1.0 - omega_m - omega_l) / (a * a) + omega_l > 0)) return GREEM_ERR_INVALID_ARG;
    }
    *kick = cosmo_integral(a0, a1, omega_m, omega_l, h0, 2);
    *drift = cosmo_integral(a0, a1, omega_m, omega_l, h0, 3);
    return GREEM_OK;
}

int greem_peak_tflops(greem_ctx *c, int which, double *tflops)
{
    if (!c || !tflops || which < 0 || which > 2) return GREEM_ERR_INVALID_ARG;
    int err = 0;
    *tflops = peak_tflops(which, c->nsm, c->stream, &err);
    return err;
}

// ------------------------------------------------------------------ domains and LETs
static bool boxes_valid(const int32_t *boxes, int ndom)
{
    for (int d = 0; d < ndom; d++)
        for (int a = 0; a < 3; a++) {
            const int32_t lo = boxes[6 * d + 2 * a], hi = boxes[6 * d + 2 * a + 1];
            if (lo < 0 || hi > (1 << 21) || lo > hi) return false;
        }
    return true;
}

int greem_cell_index(greem_ctx *c, const double *pos, int64_t N, double L, const int64_t *idx, int64_t n,
                     int32_t *cells)
{
    if (!c || !pos || !cells || N < 1 || N >= (int64_t)0x7FFFFFF0 || n < 0 || n >= (int64_t)0x7FFFFFF0 ||
        (!idx && n > N) || !(L > 0) || !std::isfinite(L))
        return GREEM_ERR_INVALID_ARG;
    if (n == 0) return GREEM_OK;
    int rc;
    if ((rc = ensure(c, c->st, 1))) return rc;
    greem_params p;
    greem_params_default(&p);
    p.L = L;
    p.r_cut = 0.25 * L;
    BoxPar bp;
    if ((rc = derive_box(p, 0, 0, bp, false))) return rc;
    greem::g_launches = 0;
    cudaStream_t s = c->stream;
    if (!cuda_ok(cudaMemsetAsync(c->st.p, 0, sizeof(DevStatus), s))) return GREEM_ERR_CUDA;
    launch_cells(pos, (uint32_t)N, idx, (uint32_t)n, L, bp.pow2_e, cells, c->st.p, s);
    unsigned flags = 0;
    if (!cuda_ok(cudaGetLastError()) ||
        !cuda_ok(cudaMemcpyAsync(&flags, &c->st.p->flags, sizeof(flags), cudaMemcpyDeviceToHost, s)) ||
        !cuda_ok(cudaStreamSynchronize(s)))
        return GREEM_ERR_CUDA;
    c->stats.kernel_launches = greem::g_launches;
    return (flags & ST_NONFINITE) ? GREEM_ERR_INVALID_ARG : GREEM_OK;
}

int greem_domain_pack(greem_ctx *c, const double *pos, const float *mass, const int64_t *ids, int64_t N, double L,
                      const int32_t *boxes, int ndom, int64_t *counts, double *pos_out, float *mass_out,
                      int64_t *ids_out)
{
    if (!c || !boxes || !counts || ndom < 1 || ndom > kMaxDomains || N < 0 || N >= (int64_t)0x7FFFFFF0 ||
        !(L > 0) || !std::isfinite(L) || !boxes_valid(boxes, ndom))
        return GREEM_ERR_INVALID_ARG;
    for (int d = 0; d < ndom; d++) counts[d] = 0;
    if (N == 0) return GREEM_OK;
    if (!pos || !mass || !pos_out || !mass_out || !ids_out) return GREEM_ERR_INVALID_ARG;
    greem_params p;
    greem_params_default(&p);
    p.L = L;
    p.r_cut = 0.25 * L;
    BoxPar bp;
    int rc;
    if ((rc = derive_box(p, 0, 0, bp, false))) return rc;
    const uint32_t n = (uint32_t)N, nblk = dom_blocks(n);
    const size_t ncnt = (size_t)ndom * nblk;
    if ((rc = ensure(c, c->st, 1)) || (rc = ensure(c, c->dom_boxes, (size_t)ndom * 6)) || (rc = ensure(c, c->dom, n)) ||
        (rc = ensure(c, c->dom_cnt, ncnt + 1)) || (rc = ensure(c, c->scratch, scan_scratch_elems(ncnt + 1) + 64)))
        return rc;
    greem::g_launches = 0;
    cudaStream_t s = c->stream;
    if (!cuda_ok(cudaMemsetAsync(c->st.p, 0, sizeof(DevStatus), s)) ||
        !cuda_ok(cudaMemcpyAsync(c->dom_boxes.p, boxes, sizeof(int32_t) * 6 * ndom, cudaMemcpyHostToDevice, s)))
        return GREEM_ERR_CUDA;
    launch_dom_count(pos, n, L, bp.pow2_e, c->dom_boxes.p, ndom, c->dom.p, c->dom_cnt.p, c->st.p, s);
    scan_u32(c->dom_cnt.p, c->dom_cnt.p, ncnt, c->scratch.p, s);
    launch_dom_scatter(pos, mass, ids, n, L, c->dom.p, c->dom_cnt.p, ndom, pos_out, mass_out, ids_out, s);
    std::vector<uint32_t> off(ncnt + 1);
    unsigned flags = 0;
    if (!cuda_ok(cudaGetLastError()) ||
        !cuda_ok(cudaMemcpyAsync(off.data(), c->dom_cnt.p, sizeof(uint32_t) * (ncnt + 1), cudaMemcpyDeviceToHost, s)) ||
        !cuda_ok(cudaMemcpyAsync(&flags, &c->st.p->flags, sizeof(flags), cudaMemcpyDeviceToHost, s)) ||
        !cuda_ok(cudaStreamSynchronize(s)))
        return GREEM_ERR_CUDA;
    c->stats.kernel_launches = greem::g_launches;
    if (flags & ST_NONFINITE) return GREEM_ERR_INVALID_ARG;
    for (int d = 0; d < ndom; d++) counts[d] = (int64_t)off[(size_t)(d + 1) * nblk] - (int64_t)off[(size_t)d * nblk];
    return GREEM_OK;
}

int greem_let_export(greem_ctx *c, const int32_t *boxes, int ndom, int self, int64_t *counts, double *pos_out,
                     float *mass_out, int64_t *ref_out, int64_t cap, int64_t *total)
{
    if (!c || !boxes || !counts || !total || ndom < 1 || ndom > kMaxDomains || self >= ndom || cap < 0 ||
        !boxes_valid(boxes, ndom))
        return GREEM_ERR_INVALID_ARG;
    *total = 0;
    if (!c->have_tree || c->last_nbox != 1) return GREEM_ERR_INVALID_ARG;
    if (cap > 0 && (!pos_out || !mass_out)) return GREEM_ERR_INVALID_ARG;
    const uint32_t N = c->last_N;
    const uint32_t ncap = (uint32_t)std::min<size_t>(c->node_cap, 0xFFFFFFF0u);
    // the receiving boxes: every box but self and the empty ones
    std::vector<int> recv;
    std::vector<LetBox> lb;
    for (int d = 0; d < ndom; d++) {
        counts[d] = 0;
        LetBox b;
        for (int a = 0; a < 3; a++) {
            const long long lo = boxes[6 * d + 2 * a], hi = boxes[6 * d + 2 * a + 1];
            b.c[a] = lo + hi;  // [2 lo, 2 hi) in u
            b.h[a] = hi - lo;
        }
        if (d == self || b.h[0] == 0 || b.h[1] == 0 || b.h[2] == 0) continue;  // an empty box imports nothing
        recv.push_back(d);
        lb.push_back(b);
    }
    const int nrecv = (int)recv.size();
    const int chunk = std::min(nrecv, kLetChunk);
    const size_t run = (size_t)ncap + 1;
    int rc;
    if (chunk > 0 &&
        ((rc = ensure(c, c->let_flag, ncap)) || (rc = ensure(c, c->let_cnt, run * chunk + 1)) ||
         (rc = ensure(c, c->let_ends, (size_t)kLetChunk + 1)) ||
         (rc = ensure(c, c->scratch, scan_scratch_elems(run * chunk + 1) + 64))))
        return rc;
    const uint32_t *n_nodes = c->base.p + N;
    cudaStream_t s = c->stream;
    greem::g_launches = 0;
    int64_t run_items = 0;
    for (int j0 = 0; j0 < nrecv; j0 += kLetChunk) {
        const int nb = std::min(kLetChunk, nrecv - j0);
        launch_let_count(c->nodes.p, n_nodes, ncap, lb.data() + j0, nb, c->bps.p, c->pcell.p, c->let_flag.p,
                         c->let_cnt.p, s, c->nsm);
        scan_u32(c->let_cnt.p, c->let_cnt.p, run * nb, c->scratch.p, s);
        launch_let_ends(c->let_cnt.p, ncap, nb, c->let_ends.p, s);
        uint32_t ends[kLetChunk + 1];
        if (!cuda_ok(cudaGetLastError()) ||
            !cuda_ok(cudaMemcpyAsync(ends, c->let_ends.p, sizeof(uint32_t) * (nb + 1), cudaMemcpyDeviceToHost, s)) ||
            !cuda_ok(cudaStreamSynchronize(s)))
            return GREEM_ERR_CUDA;
        for (int j = 0; j < nb; j++) counts[recv[j0 + j]] = (int64_t)ends[j + 1] - (int64_t)ends[j];
        const int64_t tot = ends[nb];
        if (run_items + tot <= cap && tot)
            launch_let_fill(c->nodes.p, n_nodes, ncap, lb.data() + j0, nb, c->bps.p, c->pcell.p, c->let_flag.p,
                            c->let_cnt.p, c->xs.p, c->ys.p, c->zs.p, c->ms.p, c->mom64.p, pos_out, mass_out, ref_out,
                            (unsigned long long)run_items, s, c->nsm);
        run_items += tot;
    }
    *total = run_items;
    if (!cuda_ok(cudaGetLastError()) || !cuda_ok(cudaStreamSynchronize(s))) return GREEM_ERR_CUDA;
    c->stats.kernel_launches = greem::g_launches;
    return run_items > cap ? GREEM_ERR_CAPACITY : GREEM_OK;
}

int greem_debug_set(greem_ctx *c, int what, int64_t value)
{
    if (!c) return GREEM_ERR_INVALID_ARG;
    drop_auto_graph(c);  // every setting below changes what a call enqueues
    switch (what) {
    case GREEM_DEBUG_WAIT_POLLS:
        if (value > (int64_t)kWaitPolls) return GREEM_ERR_INVALID_ARG;
        c->wait_polls1 = value < 0 ? 0u : (uint32_t)value + 1u;
        return GREEM_OK;
    case GREEM_DEBUG_NODE_CAP:
        if (value < 1 || value > (int64_t)0xFFFFFFF0) return GREEM_ERR_INVALID_ARG;
        c->next_node_cap = (size_t)value;
        return GREEM_OK;
    case GREEM_DEBUG_LIST_CAP:
        if (value < 1) return GREEM_ERR_INVALID_ARG;
        c->next_list_cap = (size_t)value;
        return GREEM_OK;
    case GREEM_DEBUG_STACK_CAP:
        if (value < 1 || value > (1 << 24)) return GREEM_ERR_INVALID_ARG;
        c->next_stack_cap = (uint32_t)value;
        return GREEM_OK;
    case GREEM_DEBUG_MAX_ATTEMPTS:
        if (value > 64) return GREEM_ERR_INVALID_ARG;
        c->max_attempts = value < 1 ? 6 : (int)value;
        return GREEM_OK;
    case GREEM_DEBUG_START_LEVEL:
        if (value > 7) return GREEM_ERR_INVALID_ARG;
        c->start_cap = value < 0 ? 7 : (int)value;
        return GREEM_OK;
    case GREEM_DEBUG_REPLAY:
        if (value < 0 || value > 1) return GREEM_ERR_INVALID_ARG;
        c->ag_enabled = value != 0;
        return GREEM_OK;
    default:
        return GREEM_ERR_INVALID_ARG;
    }
}

const char *greem_strerror(int code)
{
    switch (code) {
    case GREEM_OK: return "ok";
    case GREEM_ERR_INVALID_ARG: return "invalid argument (bad size or parameter, or a NaN/Inf position)";
    case GREEM_ERR_CUDA: return "CUDA runtime error";
    case GREEM_ERR_OOM: return "out of memory";
    case GREEM_ERR_CAPACITY: return "device buffer capacity exceeded (capture the graph again)";
    case GREEM_ERR_TIMEOUT: return "bounded device wait timed out";
    case GREEM_ERR_NOT_IMPLEMENTED: return "not implemented";
    default: return "unknown error";
    }
}

}  // extern "C"
