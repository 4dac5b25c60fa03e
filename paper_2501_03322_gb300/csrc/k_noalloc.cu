// tw_mag_noalloc: the tw_mag computation for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc at all: code running inside a CUDA
// graph capture, applications whose device memory is owned by a pool or
// arena that the library cannot see, or real-time loops where an allocation
// could stall or fail at an arbitrary moment.  This entry point runs the same
// contour-integration kernel as tw_mag, but its scratch (the work counter and
// the per-warp sample arenas) lives in a file-scope static device array that
// every GPU which loads this library holds until the process exits.
//
// Limits: NOALLOC_SLOTS warp arenas of at most NOALLOC_MAX_SAMPLES limb
// samples each (about 53 MiB per GPU), i.e. one CTA of four warps per SM on a
// 152-SM GB300 (tw_mag runs two), and a queue of NOALLOC_RELIST positions for
// the slope-repair pass.  Requests for a larger sample cap are rejected with
// TW_ETOOBIG.  All calls share the one array, which keeps the previous call's
// contents: the work counter and the repair-queue length are cleared by every
// call, the arenas and the queue entries need no clearing (each is written
// before it is read).  Calls that overlap on the GPU (on different streams,
// or racing host threads) race on the array and corrupt each other's results.
#include <mutex>

#include "../../include/twinkle.h"
#include "kernels.cuh"
#include "ptrkind.cuh"

namespace tw {

constexpr int NOALLOC_SLOTS = 608;          // 152 CTAs of 4 warps
constexpr int NOALLOC_MAX_SAMPLES = 512;
constexpr size_t NOALLOC_SLOT_BYTES = arena_slot_bytes(NOALLOC_MAX_SAMPLES);
static_assert(NOALLOC_SLOT_BYTES == 92160, "arena layout changed");
constexpr size_t NOALLOC_HEADER = 256;        // work counter, work statistics, repair-queue counters
constexpr int NOALLOC_RELIST = 4096;          // positions queued for the slope-repair pass
constexpr size_t NOALLOC_RELIST_BYTES = NOALLOC_RELIST * sizeof(int64_t);
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + NOALLOC_RELIST_BYTES + NOALLOC_SLOT_BYTES * NOALLOC_SLOTS;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

static std::mutex g_na_mu;
static char *g_na_ptr[64];  // device address of g_noalloc_scratch, per device
static int g_na_nsm[64];

// Once per device, with that device current: the device address of the static
// array (in host code its name is only a host-side stand-in).
static int noalloc_setup(int dev, char **ptr, int *nsm) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) { (void)cudaGetLastError(); return TW_ECUDA; }
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) { (void)cudaGetLastError(); return TW_ECUDA; }
        g_na_ptr[dev] = (char *)p;
        g_na_nsm[dev] = n;
    }
    *ptr = g_na_ptr[dev];
    *nsm = g_na_nsm[dev];
    return TW_OK;
}

// device (or managed) memory of the current device
static bool on_device(const void *p) { return ptr_kind(p) == PK_DEV; }

}  // namespace tw

extern "C" int tw_mag_noalloc(double s, double q, double rho, const double *y1, const double *y2, int64_t n,
                              double rel_tol, double *out, int precision, int max_samples, void *stream) {
    using namespace tw;
    auto fin = [](double v) { return isfinite(v) && v > 0.0; };
    if (n < 0 || !fin(s) || !fin(q) || !fin(rho) || !fin(rel_tol)) return TW_EINVAL;
    if (precision != TW_PREC_FP64 && precision != TW_PREC_MIXED) return TW_EINVAL;
    if (max_samples < 64) return TW_EINVAL;
    if (max_samples > NOALLOC_MAX_SAMPLES) return TW_ETOOBIG;
    if (n == 0) return TW_OK;
    if (!y1 || !y2 || !out || !on_device(y1) || !on_device(y2) || !on_device(out)) return TW_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { (void)cudaGetLastError(); return TW_ECUDA; }
    char *base = nullptr;
    int nsm = 0;
    int rc = noalloc_setup(dev, &base, &nsm);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t (*lf)(unsigned, cudaStream_t, const KParams &) =
        precision == TW_PREC_FP64 ? launch_contour_0_2 : launch_contour_1_2;
    cudaError_t (*of)(int *) = precision == TW_PREC_FP64 ? occupancy_contour_0_2 : occupancy_contour_1_2;
    int occ = 1;
    if (of(&occ) != cudaSuccess) { (void)cudaGetLastError(); return TW_ECUDA; }
    int64_t blocks = (int64_t)nsm * (occ < 1 ? 1 : occ);
    if (blocks > NOALLOC_SLOTS / WPB) blocks = NOALLOC_SLOTS / WPB;
    const int64_t need = (n + WPB - 1) / WPB;
    if (blocks > need) blocks = need;
    KParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.src.kind = 0;
    kp.src.n = n;
    kp.src.s = s;
    kp.src.q = q;
    kp.src.rho = rho;
    kp.src.y1 = y1;
    kp.src.y2 = y2;
    kp.src.stride = 1;
    kp.out = out;
    kp.arena = base + NOALLOC_HEADER + NOALLOC_RELIST_BYTES;
    kp.slot_bytes = NOALLOC_SLOT_BYTES;
    kp.cap = (max_samples + 63) & ~63;
    kp.tol = rel_tol;
    kp.chunk = 1;
    kp.counter = (unsigned long long *)base;
    // crossings that fail the slope test (Sec. 2.4.2) queue their position
    // here; the repair pass integrates them again (positions beyond the
    // queue's length keep the main pass's result)
    kp.relist = (int64_t *)(base + NOALLOC_HEADER);
    kp.relist_cap = NOALLOC_RELIST;
    // the work counter and the queue length must start at zero; the arenas
    // and the queue entries need no clearing
    if (cudaMemsetAsync(base, 0, NOALLOC_HEADER, st) != cudaSuccess) { (void)cudaGetLastError(); return TW_ECUDA; }
    if (lf((unsigned)blocks, st, kp) != cudaSuccess) { (void)cudaGetLastError(); return TW_ECUDA; }
    // the repair pass: at most one CTA per SM and never more warps than arenas
    const unsigned rblocks = (unsigned)(blocks < nsm ? blocks : nsm);
    if ((precision == TW_PREC_FP64 ? launch_repair_0 : launch_repair_1)(rblocks, st, kp) != cudaSuccess) {
        (void)cudaGetLastError();
        return TW_ECUDA;
    }
    return TW_OK;
}
