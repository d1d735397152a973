// greem_pair_force_f32_noalloc: the pairwise FP32 force of greem_pair_force_f32 for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted, e.g. a
// host library whose allocator policy forbids driver allocations, a caller that must
// not be held up by the device-wide synchronisation that cudaMalloc and cudaFree can
// impose (this call waits only for its own stream, to read its status word), or a
// process that has handed all free device memory to another allocator.  Such callers
// still own the inputs and the output; only the scratch is provided here.
//
// The scratch (one-pair groups, their padded one-entry lists, the identity permutation
// and a status word) lives in one file-scope __device__ array sized for
// kNoAllocMaxPairs pairs.  Every GPU that loads the library holds that array until the
// process exits.  Host code may not use the array's name as a device address: on the
// first call on each device, with that device current, the entry point asks the
// runtime for the array's device address (cudaGetSymbolAddress) and keeps it.  That
// first call should therefore come before any stream capture.  All calls on a device
// share the array and it keeps the last call's contents; the parts that must start at
// zero are cleared by each call.  Two calls whose work overlaps on the GPU race on the
// array, so serialise them (one stream, or wait between calls).
#include <mutex>

#include "common.cuh"
#include "greem.h"

namespace greem {

constexpr int64_t kNoAllocMaxPairs = 32768;

// byte offsets of the pieces inside the scratch array (each 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffStatus = 0;
constexpr size_t kOffBox = align256(kOffStatus + sizeof(DevStatus));
constexpr size_t kOffNGroups = align256(kOffBox + sizeof(BoxPar));
constexpr size_t kOffGroups = align256(kOffNGroups + sizeof(uint32_t));
constexpr size_t kOffIrel = align256(kOffGroups + sizeof(Group) * kNoAllocMaxPairs);
constexpr size_t kOffList = align256(kOffIrel + sizeof(float4) * kNoAllocMaxPairs);
constexpr size_t kOffLoff = align256(kOffList + sizeof(float4) * 8 * kNoAllocMaxPairs);
constexpr size_t kOffLlen = align256(kOffLoff + sizeof(unsigned long long) * kNoAllocMaxPairs);
constexpr size_t kOffLraw = align256(kOffLlen + sizeof(uint32_t) * kNoAllocMaxPairs);
constexpr size_t kOffPerm = align256(kOffLraw + sizeof(uint32_t) * kNoAllocMaxPairs);
constexpr size_t kScratchBytes = align256(kOffPerm + sizeof(uint32_t) * kNoAllocMaxPairs);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Writes the one box of constants the force kernel reads (no host staging buffer) and
// clears the status word (flags and work-queue counters), which must start at zero on
// every call.
__global__ void k_noalloc_box(BoxPar *bp, DevStatus *st, float inv_rc2, float eps2)
{
    if (threadIdx.x == 0) {
        BoxPar b = {};
        b.inv_rc2 = inv_rc2;
        b.eps2 = eps2;
        *bp = b;
    }
    uint32_t *w = reinterpret_cast<uint32_t *>(st);
    for (int i = threadIdx.x; i < (int)(sizeof(DevStatus) / 4); i += blockDim.x) w[i] = 0u;
}

static int launch_failed()
{
    return cudaGetLastError() != cudaSuccess;
}

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[256];

}  // namespace greem

using namespace greem;

extern "C" int greem_pair_force_f32_noalloc(const double *x_g, const double *x_i, const double *x_j, const float *m_j,
                                            int64_t npairs, double r_cut, double eps, float *acc, void *cuda_stream)
{
    if (!x_g || !x_i || !x_j || !m_j || !acc) return GREEM_ERR_INVALID_ARG;
    if (npairs < 1 || npairs > kNoAllocMaxPairs || !(r_cut > 0) || !(eps >= 0)) return GREEM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return GREEM_ERR_CUDA;
    }
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return GREEM_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DevStatus *st = reinterpret_cast<DevStatus *>(base + kOffStatus);
    BoxPar *bp = reinterpret_cast<BoxPar *>(base + kOffBox);
    uint32_t *ng = reinterpret_cast<uint32_t *>(base + kOffNGroups);
    Group *groups = reinterpret_cast<Group *>(base + kOffGroups);
    float4 *irel = reinterpret_cast<float4 *>(base + kOffIrel);
    float4 *flist = reinterpret_cast<float4 *>(base + kOffList);
    unsigned long long *loff = reinterpret_cast<unsigned long long *>(base + kOffLoff);
    uint32_t *llen = reinterpret_cast<uint32_t *>(base + kOffLlen);
    uint32_t *lraw = reinterpret_cast<uint32_t *>(base + kOffLraw);
    uint32_t *perm = reinterpret_cast<uint32_t *>(base + kOffPerm);

    const double inv_rc = 1.0 / r_cut;
    // an error left by earlier work on this thread is not this call's
    cudaGetLastError();
    k_noalloc_box<<<1, 32, 0, s>>>(bp, st, (float)(inv_rc * inv_rc), (float)((eps / r_cut) * (eps / r_cut)));
    if (launch_failed()) return GREEM_ERR_CUDA;
    launch_pair_setup(x_g, x_i, x_j, m_j, (uint32_t)npairs, inv_rc, groups, irel, flist, loff, llen, lraw, perm, ng,
                      s);
    if (launch_failed()) return GREEM_ERR_CUDA;
    ForceArgs fa = {};
    fa.groups = groups;
    fa.n_groups = ng;
    fa.order = nullptr;
    fa.loff = loff;
    fa.llen = llen;
    fa.lraw = lraw;
    fa.flist = flist;
    fa.irel = irel;
    fa.perm = perm;
    fa.bps = bp;
    fa.acc = acc;
    fa.st = st;
    fa.chunk = 256;
    fa.warps = 8;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return GREEM_ERR_CUDA;
    }
    launch_force_f32(fa, s, nsm, eps > 0);
    if (launch_failed()) return GREEM_ERR_CUDA;
    unsigned int flags = 0;
    if (cudaMemcpyAsync(&flags, &st->flags, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return GREEM_ERR_CUDA;
    }
    if (flags & ST_TIMEOUT) return GREEM_ERR_TIMEOUT;
    return GREEM_OK;
}
