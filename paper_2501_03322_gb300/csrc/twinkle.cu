// twinkle.cu -- launch runtime and C ABI of libtwinkle_gb300.so (host code).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <stdio.h>
#include <stdlib.h>
#include <sys/stat.h>

#include <map>
#include <mutex>
#include <string>

#include "../../include/twinkle.h"
#include "kernels.cuh"
#include "ptrkind.cuh"

namespace tw {

// ---------------------------------------------------------------- runtime

typedef cudaError_t (*launch_fn)(unsigned, cudaStream_t, const KParams &);
typedef cudaError_t (*occ_fn)(int *);

static void pick_kernel(int prec, int spl, bool occ4, int w, launch_fn *lf, occ_fn *of) {
    if (w == 2) {
        if (prec == 0) { *lf = launch_contour_0_w2; *of = occupancy_contour_0_w2; }
        else { *lf = launch_contour_1_w2; *of = occupancy_contour_1_w2; }
        return;
    }
    if (w == 4) {
        if (prec == 0) { *lf = launch_contour_0_w4; *of = occupancy_contour_0_w4; }
        else { *lf = launch_contour_1_w4; *of = occupancy_contour_1_w4; }
        return;
    }
    if (spl == 2 && occ4) {
        if (prec == 0) { *lf = launch_contour_0_2_o4; *of = occupancy_contour_0_2_o4; }
        else { *lf = launch_contour_1_2_o4; *of = occupancy_contour_1_2_o4; }
        return;
    }
    if (prec == 0) {
        if (spl == 1) { *lf = launch_contour_0_1; *of = occupancy_contour_0_1; }
        else if (spl == 2) { *lf = launch_contour_0_2; *of = occupancy_contour_0_2; }
        else { *lf = launch_contour_0_4; *of = occupancy_contour_0_4; }
    } else {
        if (spl == 1) { *lf = launch_contour_1_1; *of = occupancy_contour_1_1; }
        else if (spl == 2) { *lf = launch_contour_1_2; *of = occupancy_contour_1_2; }
        else { *lf = launch_contour_1_4; *of = occupancy_contour_1_4; }
    }
}

struct DevState {
    bool init = false;
    int nsm = 0;
    char *arena = nullptr;
    size_t arena_bytes = 0;
    unsigned long long *counter = nullptr;
    char *stage = nullptr;          // device staging for host-pointer calls
    size_t stage_bytes = 0;
    cudaEvent_t last = nullptr;     // completion of the previous launch (serialises calls)
    cudaEvent_t t0 = nullptr, t1 = nullptr;  // timing events around the latest kernel launch
    bool timed = false;             // t0/t1 hold a launch
    int64_t *relist = nullptr;      // work items queued for the slope-repair pass
    size_t relist_bytes = 0;
    char *calib = nullptr;          // outputs of autotuning calibration runs
    size_t calib_bytes = 0;
    cudaGraphExec_t graph = nullptr;  // replayable {counter reset, persistent kernel}
    char *ld = nullptr;             // node scratch of the limb-darkening kernel
    size_t ld_bytes = 0;
    char name[256] = {0};           // device name (autotune cache key)
};

static std::mutex g_mu;
static DevState g_dev[64];

static int cuda_fail(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TW_ENOMEM : TW_ECUDA;
}

static int dev_state(DevState **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= 64) return TW_ECUDA;
    DevState &d = g_dev[dev];
    if (!d.init) {
        if ((e = cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaMalloc(&d.counter, 64)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaEventCreateWithFlags(&d.last, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaEventCreate(&d.t0)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaEventCreate(&d.t1)) != cudaSuccess) return cuda_fail(e);
        cudaDeviceProp prop;
        if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) return cuda_fail(e);
        snprintf(d.name, sizeof(d.name), "%s", prop.name);
        d.init = true;
    }
    *out = &d;
    return TW_OK;
}

// Optional cap on the library's device working memory, in bytes
// ($TW_DEVICE_MEMORY_LIMIT; unset or 0: no cap): a request beyond it fails
// with TW_ENOMEM as a failed cudaMalloc would, before anything is freed or
// allocated.  It lets callers bound the library's footprint and lets tests
// make an allocation fail without exhausting a GPU.
static size_t memory_limit() {
    const char *v = getenv("TW_DEVICE_MEMORY_LIMIT");
    if (!v || !*v) return 0;
    return (size_t)strtoull(v, nullptr, 10);
}

static int grow(char **buf, size_t *have, size_t need) {
    if (*have >= need) return TW_OK;
    const size_t lim = memory_limit();
    if (lim && need > lim) return TW_ENOMEM;
    if (*buf) {
        cudaDeviceSynchronize();
        cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
    }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) { *buf = nullptr; return cuda_fail(e); }
    *have = need;
    return TW_OK;
}


static bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

static int check_opts(const tw_opts *o) {
    if (!o) return TW_OK;
    if (o->precision != TW_PREC_FP64 && o->precision != TW_PREC_MIXED) return TW_EINVAL;
    const int spi = o->samples_per_iter;
    if (spi != 32 && spi != 64 && spi != 128) return TW_EINVAL;
    if (o->max_samples < 64 || o->max_samples > 16384 || o->max_samples < spi) return TW_EINVAL;
    const int w = o->warps_per_position;
    if (w != 0 && w != 1 && w != 2 && w != 4) return TW_EINVAL;
    if (o->max_samples < 32 * (w > 1 ? w : 1)) return TW_EINVAL;
    return TW_OK;
}

// Launch shape: samples per lane per iteration, CTAs per SM (0: as many as
// fit), work items per atomic grab, which compiled instance (occ4 = 1 the one
// built for 4 CTAs per SM (spl 2 only), 0 the one built for 2, -1 by work
// kind: see launch()), and w, the warps that integrate each position together
// (1; or 2 or 4 with one sample per lane).  Limb samples per iteration =
// 32 x spl x w.
struct LaunchCfg {
    int spl, ctas, chunk, occ4, w;
};

// Launches the contour kernel over src.n positions.  Device pointers only.
// With use_graph the counter reset and the kernel are replayed from a CUDA
// graph (captured on the call's stream and updated in place on later calls)
// instead of being launched one by one.
static int launch(DevState &d, WorkSrc src, double tol, int prec, int max_samples, LaunchCfg cfg, bool use_graph,
                  double *out, double *err, int32_t *nsamp, int8_t *pstat, cudaStream_t st) {
    const int cap = (max_samples + 63) & ~63;
    if (src.stride < 1) src.stride = 1;
    launch_fn lf;
    occ_fn of;
    int w = (cfg.w == 2 || cfg.w == 4) ? cfg.w : 1;
    // per-position lenses, untuned, at 64 samples per iteration: two warps
    // per position (measured on 2^18 queries near caustics, mixed precision:
    // 136 ms, against 149 ms for the 4-CTA instance and 177 ms for one warp
    // per position)
    if (w == 1 && cfg.occ4 < 0 && src.kind == 3 && cfg.spl == 2) {
        w = 2;
        cfg.spl = 1;
    }
    const bool occ4 = w == 1 && (cfg.occ4 > 0 || (cfg.occ4 < 0 && src.kind == 3));
    pick_kernel(prec, cfg.spl, occ4, w, &lf, &of);
    if (src.kind == 5) {  // limb-darkened sources: their own kernel, one warp per source
        w = 1;
        if (prec == 0) { lf = launch_ld_0; of = occupancy_ld_0; }
        else { lf = launch_ld_1; of = occupancy_ld_1; }
    }
    int occ = 0;
    cudaError_t e = of(&occ);
    if (e != cudaSuccess) return cuda_fail(e);
    if (occ < 1) occ = 1;
    if (cfg.ctas > 0 && cfg.ctas < occ) occ = cfg.ctas;
    int64_t blocks = (int64_t)d.nsm * occ;
    const int per_cta = WPB / w;  // positions in flight per CTA
    const int64_t need_blocks = (src.n + per_cta - 1) / per_cta;
    if (blocks > need_blocks) blocks = need_blocks;
    if (blocks < 1) blocks = 1;
    const size_t slot_bytes = arena_slot_bytes(cap);
    int rc = grow(&d.arena, &d.arena_bytes, slot_bytes * (size_t)blocks * WPB);
    if (rc) return rc;
    if (src.kind == 5 && (rc = grow(&d.ld, &d.ld_bytes, (size_t)blocks * WPB * LD_WARP_DOUBLES * sizeof(double))))
        return rc;
    // repair queue: room for every work item up to 2^20 (positions beyond it
    // that fail the slope test keep the main pass's result and PS_SLOPE)
    const size_t relist_cap = (size_t)(src.n < (1 << 20) ? (src.n > 0 ? src.n : 1) : (1 << 20));
    if ((rc = grow((char **)&d.relist, &d.relist_bytes, relist_cap * sizeof(int64_t)))) return rc;
    // serialise with the previous launch (the arena and counter are shared)
    if ((e = cudaStreamWaitEvent(st, d.last, 0)) != cudaSuccess) return cuda_fail(e);
    KParams kp;
    kp.src = src;
    kp.out = out;
    kp.err = err;
    kp.nsamp = nsamp;
    kp.pstat = pstat;
    kp.arena = d.arena;
    kp.slot_bytes = slot_bytes;
    kp.cap = cap;
    kp.tol = tol;
    kp.chunk = cfg.chunk < 1 ? 1 : cfg.chunk;
    kp.counter = d.counter;
    kp.relist = d.relist;
    kp.relist_cap = d.relist_bytes / sizeof(int64_t);
    kp.ld = (double *)d.ld;
    // main pass, then the repair pass over the items it queued (usually none:
    // the repair kernel finds an empty queue and exits)
    auto kernels = [&]() -> cudaError_t {
        cudaError_t e0 = lf((unsigned)blocks, st, kp);
        if (e0 != cudaSuccess) return e0;
        // at most one CTA per SM (one four-warp group and one arena slot each)
        const unsigned rblocks = (unsigned)(blocks < d.nsm ? blocks : d.nsm);
        return (prec == TW_PREC_FP64 ? launch_repair_0 : launch_repair_1)(rblocks, st, kp);
    };
    bool graphed = false;
    if (use_graph && st != nullptr) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaMemsetAsync(d.counter, 0, 8 * sizeof(unsigned long long), st);
            cudaError_t e2 = kernels();
            e = cudaStreamEndCapture(st, &g);
            if (e == cudaSuccess && e1 == cudaSuccess && e2 == cudaSuccess) {
                bool ok = false;
                if (d.graph) {
                    cudaGraphExecUpdateResultInfo info;
                    ok = cudaGraphExecUpdate(d.graph, g, &info) == cudaSuccess;
                    if (!ok) { (void)cudaGetLastError(); cudaGraphExecDestroy(d.graph); d.graph = nullptr; }
                }
                if (!ok) ok = cudaGraphInstantiate(&d.graph, g, 0) == cudaSuccess;
                if (ok) {
                    d.timed = cudaEventRecord(d.t0, st) == cudaSuccess;
                    graphed = cudaGraphLaunch(d.graph, st) == cudaSuccess;
                    d.timed = d.timed && graphed && cudaEventRecord(d.t1, st) == cudaSuccess;
                }
            }
            if (g) cudaGraphDestroy(g);
        }
        (void)cudaGetLastError();
    }
    if (!graphed) {
        if ((e = cudaMemsetAsync(d.counter, 0, 8 * sizeof(unsigned long long), st)) != cudaSuccess) return cuda_fail(e);
        d.timed = cudaEventRecord(d.t0, st) == cudaSuccess;
        if ((e = kernels()) != cudaSuccess) { d.timed = false; return cuda_fail(e); }
        d.timed = d.timed && cudaEventRecord(d.t1, st) == cudaSuccess;
    }
    (void)cudaGetLastError();
    if ((e = cudaEventRecord(d.last, st)) != cudaSuccess) return cuda_fail(e);
    return TW_OK;
}

// ---------------------------------------------------------------- autotuner
//
// Chooses the launch shape by timing a calibration sub-sample (every k-th
// position, about 5% of the call, at least 16 positions per resident warp and
// at most 65536) for every
// candidate, and caches the fastest per (GPU name, precision, tolerance
// decade, workload kind) in memory and in a small text file
// ($TW_AUTOTUNE_CACHE, default $HOME/.cache/twinkle_gb300_autotune.txt).
// The samples per iteration it picks change the limb sampling, so results
// differ from an untuned call within the tolerance.

static std::map<std::string, LaunchCfg> g_tune;
static bool g_tune_loaded = false;

static std::string tune_path() {
    const char *p = getenv("TW_AUTOTUNE_CACHE");
    if (p && *p) return p;
    const char *h = getenv("HOME");
    return std::string(h && *h ? h : "/tmp") + "/.cache/twinkle_gb300_autotune.txt";
}

static void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    FILE *f = fopen(tune_path().c_str(), "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        char *bar = strrchr(line, '|');
        if (!bar) continue;
        LaunchCfg c;
        c.occ4 = -1;
        c.w = 1;
        if (sscanf(bar + 1, "%d %d %d %d %d", &c.spl, &c.ctas, &c.chunk, &c.occ4, &c.w) < 3) continue;
        if (c.spl != 1 && c.spl != 2 && c.spl != 4) continue;
        if (c.w != 1 && c.w != 2 && c.w != 4) continue;
        *bar = 0;
        g_tune[line] = c;
    }
    fclose(f);
}

static void tune_save() {
    std::string path = tune_path();
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);  // may exist
    FILE *f = fopen(path.c_str(), "w");
    if (!f) return;
    for (auto &kv : g_tune)
        fprintf(f, "%s|%d %d %d %d %d\n", kv.first.c_str(), kv.second.spl, kv.second.ctas, kv.second.chunk,
                kv.second.occ4, kv.second.w);
    fclose(f);
}

static std::string tune_key(const DevState &d, int prec, double tol, int kind) {
    char buf[400];
    snprintf(buf, sizeof(buf), "%s;prec=%d;tol=1e%d;kind=%d", d.name, prec, (int)floor(log10(tol) + 1e-9), kind);
    return buf;
}

static int autotune(DevState &d, const WorkSrc &src, double tol, int prec, int max_samples, cudaStream_t st,
                    LaunchCfg *best) {
    tune_load();
    const std::string key = tune_key(d, prec, tol, src.kind);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { *best = it->second; return TW_OK; }
    // the sub-sample must give every resident warp a dozen positions or more,
    // otherwise the timing measures the tail of the launch, not its
    // throughput; a workload smaller than that is timed whole (it is then
    // tail-bound, which is what warps per position address)
    const int64_t warps = (int64_t)d.nsm * 2 * WPB;
    int64_t ncal = src.n / 20;
    if (ncal < 16 * warps) ncal = 16 * warps;
    if (ncal > 65536) ncal = 65536;
    if (ncal > src.n) ncal = src.n;
    const int64_t stride = (src.n + ncal - 1) / ncal;
    WorkSrc cal = src;
    cal.stride = stride;
    cal.n = (src.n + stride - 1) / stride;
    int rc = grow(&d.calib, &d.calib_bytes, (size_t)cal.n * 8);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
    float best_ms = 3.0e38f;
    // (samples per lane, compiled instance, warps per position): the 4-CTA
    // instance exists for 2 samples per lane, the cooperative ones for 1
    const int spls[6] = {1, 2, 4, 2, 1, 1}, occs[6] = {0, 0, 0, 1, 0, 0}, ws[6] = {1, 1, 1, 1, 2, 4};
    const int ctass[2] = {1, 0};
    const int chunks[2] = {1, 4};
    for (int a = 0; a < 6; a++)
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < 2; c++) {
                const LaunchCfg cfg = {spls[a], ctass[b], chunks[c], occs[a], ws[a]};
                float ms = 0.f;
                for (int rep = 0; rep < 2; rep++) {  // first run warms the arena and caches
                    cudaEventRecord(e0, st);
                    rc = launch(d, cal, tol, prec, max_samples, cfg, false, (double *)d.calib, nullptr, nullptr,
                                nullptr, st);
                    if (rc) break;
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = TW_ECUDA; break; }
                    cudaEventElapsedTime(&ms, e0, e1);
                }
                if (rc) break;
                if (ms < best_ms) { best_ms = ms; *best = cfg; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    g_tune[key] = *best;
    tune_save();
    return TW_OK;
}

// Runs one call: validates pointer kinds, stages host buffers, launches.
// ins/insz: input arrays (host or device) and their byte sizes; the staged
// device copies are handed to `bind`, which fills src from them.
struct Call {
    const void *in[5];
    size_t insz[5];
    int nin;
    int64_t n;  // positions (outputs)
};

template <typename Bind>
static int run_call(const Call &c, double tol, const tw_opts *opts_in, double *out, Bind bind) {
    tw_opts o;
    tw_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (check_opts(&o)) return TW_EINVAL;
    if (c.n == 0) return TW_OK;
    // the smallest sample arena any launch needs (one CTA) must fit the cap:
    // checked before any device work, so nothing is written
    const size_t lim = memory_limit();
    if (lim && arena_slot_bytes((o.max_samples + 63) & ~63) * WPB > lim) return TW_ENOMEM;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState *dp = nullptr;
    int rc = dev_state(&dp);
    if (rc) return rc;
    DevState &d = *dp;
    cudaStream_t st = (cudaStream_t)o.stream;
    // all arrays of a call must be of one kind
    // one kind for every array of the call; device memory of another device is refused
    const int kind = ptr_kind(out);
    if (kind == PK_OTHER) return TW_EINVAL;
    const bool dev = kind == PK_DEV;
    for (int i = 0; i < c.nin; i++)
        if (c.insz[i] && ptr_kind(c.in[i]) != kind) return TW_EINVAL;
    if (o.err_out && ptr_kind(o.err_out) != kind) return TW_EINVAL;
    if (o.nsamp_out && ptr_kind(o.nsamp_out) != kind) return TW_EINVAL;
    if (o.pos_status && ptr_kind(o.pos_status) != kind) return TW_EINVAL;
    const void *din[5];
    LaunchCfg cfg = {o.samples_per_iter / 32, 0, 1, -1, 1};
    if (o.warps_per_position == 2 || o.warps_per_position == 4) {
        cfg.w = o.warps_per_position;
        cfg.spl = 1;
    }
    if (dev) {
        for (int i = 0; i < c.nin; i++) din[i] = c.in[i];
        WorkSrc src = bind(din);
        if (o.autotune && src.kind != 5 && (rc = autotune(d, src, tol, o.precision, o.max_samples, st, &cfg))) return rc;
        return launch(d, src, tol, o.precision, o.max_samples, cfg, o.use_graph != 0, out, o.err_out, o.nsamp_out,
                      o.pos_status, st);
    }
    // host pointers: stage inputs and outputs through device memory
    size_t off[5], total = 0;
    for (int i = 0; i < c.nin; i++) { off[i] = total; total += align256(c.insz[i]); }
    const size_t o_out = total; total += align256((size_t)c.n * 8);
    const size_t o_err = total; total += align256((size_t)c.n * 8);
    const size_t o_ns = total; total += align256((size_t)c.n * 4);
    const size_t o_ps = total; total += align256((size_t)c.n);
    if ((rc = grow(&d.stage, &d.stage_bytes, total))) return rc;
    cudaError_t e;
    // the staging buffer is shared: wait for the previous call to finish with it
    if ((e = cudaStreamWaitEvent(st, d.last, 0)) != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < c.nin; i++) {
        din[i] = d.stage + off[i];
        if (c.insz[i] && (e = cudaMemcpyAsync(d.stage + off[i], c.in[i], c.insz[i], cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e);
    }
    WorkSrc src = bind(din);
    double *dout = (double *)(d.stage + o_out);
    double *derr = o.err_out ? (double *)(d.stage + o_err) : nullptr;
    int32_t *dns = o.nsamp_out ? (int32_t *)(d.stage + o_ns) : nullptr;
    int8_t *dps = (int8_t *)(d.stage + o_ps);
    if (o.autotune && src.kind != 5 && (rc = autotune(d, src, tol, o.precision, o.max_samples, st, &cfg))) return rc;
    if ((rc = launch(d, src, tol, o.precision, o.max_samples, cfg, o.use_graph != 0, dout, derr, dns, dps, st)))
        return rc;
    int8_t *hps = o.pos_status;
    int8_t *tmp_ps = nullptr;
    if (!hps) { tmp_ps = new int8_t[c.n]; hps = tmp_ps; }
    e = cudaMemcpyAsync(out, dout, (size_t)c.n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && derr) e = cudaMemcpyAsync(o.err_out, derr, (size_t)c.n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && dns) e = cudaMemcpyAsync(o.nsamp_out, dns, (size_t)c.n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hps, dps, (size_t)c.n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int warn = TW_OK;
    if (e == cudaSuccess)
        for (int64_t i = 0; i < c.n; i++)
            if (hps[i] & PS_CAP) { warn = TW_WCAP; break; }
    delete[] tmp_ps;
    if (e != cudaSuccess) return cuda_fail(e);
    return warn;
}

int contour_positions(const double *s, const double *q, const double *rho, const double *y1, const double *y2,
                      const int32_t *list, int64_t n, double tol, int prec, int max_samples, double *out,
                      int8_t *status, cudaStream_t st) {
    if (n == 0) return TW_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState *dp = nullptr;
    int rc = dev_state(&dp);
    if (rc) return rc;
    WorkSrc w;
    memset(&w, 0, sizeof(w));
    w.kind = 3;
    w.n = n;
    w.stride = 1;
    w.ps = s;
    w.pq = q;
    w.prho = rho;
    w.y1 = y1;
    w.y2 = y2;
    w.list = list;
    const LaunchCfg cfg = {2, 0, 1, -1, 1};
    return launch(*dp, w, tol, prec, max_samples, cfg, false, out, nullptr, nullptr, status, st);
}

}  // namespace tw

using namespace tw;

extern "C" {

void tw_opts_default(tw_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = TW_PREC_FP64;
    o->samples_per_iter = 64;
    o->max_samples = 4096;
    o->autotune = 0;
    o->warps_per_position = 1;
}

int tw_mag_ex(double s, double q, double rho, const double *y1, const double *y2, int64_t n, double rel_tol,
              double *out, const tw_opts *opts) {
    if (n < 0 || !finite_pos(s) || !finite_pos(q) || !finite_pos(rho) || !finite_pos(rel_tol)) return TW_EINVAL;
    if (n > 0 && (!y1 || !y2 || !out)) return TW_EINVAL;
    Call c;
    c.nin = 2;
    c.in[0] = y1; c.insz[0] = (size_t)n * 8;
    c.in[1] = y2; c.insz[1] = (size_t)n * 8;
    c.n = n;
    return run_call(c, rel_tol, opts, out, [&](const void **din) {
        WorkSrc w;
        memset(&w, 0, sizeof(w));
        w.kind = 0; w.n = n; w.s = s; w.q = q; w.rho = rho; w.stride = 1;
        w.y1 = (const double *)din[0];
        w.y2 = (const double *)din[1];
        return w;
    });
}

int tw_mag_ld(double s, double q, double rho, double u, const double *y1, const double *y2, int64_t n,
              double rel_tol, double *out, const tw_opts *opts) {
    if (n < 0 || !finite_pos(s) || !finite_pos(q) || !finite_pos(rho) || !finite_pos(rel_tol) || !isfinite(u) ||
        u < 0.0 || u > 1.0)
        return TW_EINVAL;
    if (n > 0 && (!y1 || !y2 || !out)) return TW_EINVAL;
    Call c;
    c.nin = 2;
    c.in[0] = y1; c.insz[0] = (size_t)n * 8;
    c.in[1] = y2; c.insz[1] = (size_t)n * 8;
    c.n = n;
    return run_call(c, rel_tol, opts, out, [&](const void **din) {
        WorkSrc w;
        memset(&w, 0, sizeof(w));
        w.kind = 5; w.n = n; w.s = s; w.q = q; w.rho = rho; w.stride = 1; w.ld_u = u;
        w.y1 = (const double *)din[0];
        w.y2 = (const double *)din[1];
        return w;
    });
}

int tw_mag(double s, double q, double rho, const double *y1, const double *y2, int64_t n, double rel_tol,
           double *out) {
    return tw_mag_ex(s, q, rho, y1, y2, n, rel_tol, out, nullptr);
}

int tw_lightcurve_ex(double s, double q, double rho, double u0, double alpha, double t0, double tE,
                     const double *times, int64_t n, double rel_tol, double *out, const tw_opts *opts) {
    if (n < 0 || !finite_pos(s) || !finite_pos(q) || !finite_pos(rho) || !finite_pos(rel_tol) || !finite_pos(tE) ||
        !isfinite(u0) || !isfinite(alpha) || !isfinite(t0))
        return TW_EINVAL;
    if (n > 0 && (!times || !out)) return TW_EINVAL;
    Call c;
    c.nin = 1;
    c.in[0] = times; c.insz[0] = (size_t)n * 8;
    c.n = n;
    return run_call(c, rel_tol, opts, out, [&](const void **din) {
        WorkSrc w;
        memset(&w, 0, sizeof(w));
        w.kind = 1; w.n = n; w.s = s; w.q = q; w.rho = rho; w.stride = 1;
        w.u0 = u0; w.alpha = alpha; w.t0 = t0; w.tE = tE;
        w.times = (const double *)din[0];
        return w;
    });
}

int tw_lightcurve_orbital(double s, double q, double rho, double u0, double alpha, double t0, double tE,
                          double ds_dt, double dalpha_dt, const double *times, int64_t n, double rel_tol, double *out,
                          const tw_opts *opts) {
    if (n < 0 || !finite_pos(s) || !finite_pos(q) || !finite_pos(rho) || !finite_pos(rel_tol) || !finite_pos(tE) ||
        !isfinite(u0) || !isfinite(alpha) || !isfinite(t0) || !isfinite(ds_dt) || !isfinite(dalpha_dt))
        return TW_EINVAL;
    if (n > 0 && (!times || !out)) return TW_EINVAL;
    Call c;
    c.nin = 1;
    c.in[0] = times; c.insz[0] = (size_t)n * 8;
    c.n = n;
    return run_call(c, rel_tol, opts, out, [&](const void **din) {
        WorkSrc w;
        memset(&w, 0, sizeof(w));
        w.kind = 4; w.n = n; w.s = s; w.q = q; w.rho = rho; w.stride = 1;
        w.u0 = u0; w.alpha = alpha; w.t0 = t0; w.tE = tE;
        w.ds_dt = ds_dt; w.dalpha_dt = dalpha_dt;
        w.times = (const double *)din[0];
        return w;
    });
}

int tw_lightcurve(double s, double q, double rho, double u0, double alpha, double t0, double tE,
                  const double *times, int64_t n, double rel_tol, double *out) {
    return tw_lightcurve_ex(s, q, rho, u0, alpha, t0, tE, times, n, rel_tol, out, nullptr);
}

int tw_mag_multi(const double *s, const double *q, const double *rho, const double *y1, const double *y2, int64_t n,
                 double rel_tol, double *out, const tw_opts *opts) {
    if (n < 0 || !finite_pos(rel_tol)) return TW_EINVAL;
    if (n > 0 && (!s || !q || !rho || !y1 || !y2 || !out)) return TW_EINVAL;
    Call c;
    c.nin = 5;
    const double *a[5] = {s, q, rho, y1, y2};
    for (int i = 0; i < 5; i++) { c.in[i] = a[i]; c.insz[i] = (size_t)n * 8; }
    c.n = n;
    return run_call(c, rel_tol, opts, out, [&](const void **din) {
        WorkSrc w;
        memset(&w, 0, sizeof(w));
        w.kind = 3; w.n = n; w.stride = 1;
        w.ps = (const double *)din[0];
        w.pq = (const double *)din[1];
        w.prho = (const double *)din[2];
        w.y1 = (const double *)din[3];
        w.y2 = (const double *)din[4];
        return w;
    });
}

int tw_lightcurve_batch(const double *params, const int64_t *offsets, const double *times, int64_t ncurve,
                        double rel_tol, double *out, const tw_opts *opts) {
    if (ncurve < 0 || !finite_pos(rel_tol)) return TW_EINVAL;
    if (ncurve == 0) return TW_OK;
    if (!params || !offsets) return TW_EINVAL;
    // the total length is needed on the host: read offsets[ncurve]
    int64_t total = 0;
    const int okind = ptr_kind(offsets);
    if (okind == PK_OTHER) return TW_EINVAL;
    if (okind == PK_DEV) {
        if (cudaMemcpy(&total, offsets + ncurve, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
    } else {
        if (offsets[0] != 0) return TW_EINVAL;
        for (int64_t k = 0; k < ncurve; k++)
            if (offsets[k + 1] < offsets[k]) return TW_EINVAL;
        total = offsets[ncurve];
    }
    if (total < 0) return TW_EINVAL;
    if (total > 0 && (!times || !out)) return TW_EINVAL;
    Call c;
    c.nin = 3;
    c.in[0] = params; c.insz[0] = (size_t)ncurve * 7 * 8;
    c.in[1] = offsets; c.insz[1] = (size_t)(ncurve + 1) * 8;
    c.in[2] = times; c.insz[2] = (size_t)total * 8;
    c.n = total;
    return run_call(c, rel_tol, opts, out, [&](const void **din) {
        WorkSrc w;
        memset(&w, 0, sizeof(w));
        w.kind = 2; w.n = total; w.stride = 1;
        w.params = (const double *)din[0];
        w.offsets = (const int64_t *)din[1];
        w.times = (const double *)din[2];
        w.ncurve = ncurve;
        return w;
    });
}

const char *tw_status_str(int code) {
    switch (code) {
        case TW_OK: return "ok";
        case TW_EINVAL: return "invalid argument";
        case TW_ECUDA: return "CUDA runtime error";
        case TW_ENOMEM: return "out of device memory";
        case TW_ETIMEOUT: return "device-side wait timed out";
        case TW_ETOOBIG: return "request exceeds the static scratch of tw_mag_noalloc (max_samples > 512)";
        case TW_WCAP: return "sample cap reached for at least one position";
        default: break;
    }
    return "unknown status";
}

int tw_version(void) { return 100; }

int tw_selftest(double *rcp_max_rel_err) {
    if (!rcp_max_rel_err) return TW_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState *dp = nullptr;
    int rc = dev_state(&dp);
    if (rc) return rc;
    unsigned long long *slot = dp->counter + 6;  // two scratch words of the control block
    cudaError_t e = cudaStreamWaitEvent(0, dp->last, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(slot, 0, 16, 0);
    if (e == cudaSuccess) e = launch_rcp_selftest(slot, 1 << 20, 0);
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, slot, 16, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    memcpy(rcp_max_rel_err, h, 16);
    return TW_OK;
}

int tw_peak_probe(int kind, double *flops_per_s) {
    if (!flops_per_s || (kind != 0 && kind != 1)) return TW_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState *dp = nullptr;
    int rc = dev_state(&dp);
    if (rc) return rc;
    if (cudaStreamWaitEvent(0, dp->last, 0) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
    return fma_probe(kind, dp->nsm, flops_per_s) ? TW_ECUDA : TW_OK;
}

int tw_last_launch_ms(float *ms) {
    if (!ms) return TW_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState *dp = nullptr;
    int rc = dev_state(&dp);
    if (rc) return rc;
    if (!dp->timed) return TW_EINVAL;
    cudaError_t e = cudaEventSynchronize(dp->t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, dp->t0, dp->t1);
    if (e != cudaSuccess) return cuda_fail(e);
    return TW_OK;
}

int tw_last_launch_work(int64_t out[5]) {
    if (!out) return TW_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState *dp = nullptr;
    int rc = dev_state(&dp);
    if (rc) return rc;
    cudaError_t e = cudaEventSynchronize(dp->last);
    unsigned long long h[6];
    if (e == cudaSuccess) e = cudaMemcpy(h, dp->counter, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < 5; i++) out[i] = (int64_t)h[i + 1];
    return TW_OK;
}

}  // extern "C"
