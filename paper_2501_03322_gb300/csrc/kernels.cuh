// kernels.cuh -- the contour-integration kernel and its work sources.
//
// Work distribution: a persistent grid (a whole number of CTAs per SM, 4
// warps each) whose warps take source positions one at a time from a global
// atomic counter (work stealing).  This replaces the paper's multi-stream
// dispatch and its re-dispatched list of unfinished sources (Sec. 3, Sec. 4.1):
// a warp that finishes a cheap position immediately takes the next one, so
// expensive caustic-crossing positions do not stall an SM.  Light curves are
// flattened into (curve, time) work items whose trajectory point is computed
// when the item is taken.
//
// Each (precision, samples-per-lane) instance is compiled in its own
// translation unit (k_*.cu) and exposed through a plain host launcher, so the
// instances build in parallel.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "contour.cuh"

namespace tw {

constexpr int TPB = 128;  // 4 warps per CTA
constexpr int WPB = TPB / 32;
#ifndef TW_MIN_CTAS_PER_SM
#define TW_MIN_CTAS_PER_SM 2  // register budget: 65536 / (128 x 2) = 256 per thread
#endif

// Where the positions of a launch come from.
struct WorkSrc {
    int kind;  // 0: one lens, arrays of positions; 1: one light curve; 2: batch of light curves;
               // 3: per-position lens (surrogate fallback and training labels);
               // 4: one light curve of an orbiting lens (s and alpha linear in time);
               // 5: one lens, arrays of positions of limb-darkened sources (ld_kernel)
    int64_t n;
    double s, q, rho;                      // kinds 0 and 1
    const double *y1, *y2;                 // kind 0
    double u0, alpha, t0, tE;              // kinds 1 and 4
    double ds_dt, dalpha_dt;               // kind 4: rates of the separation and of the binary axis angle
    double ld_u;                           // kind 5: linear limb-darkening coefficient (positions as kind 0)
    const double *times;                   // kinds 1 and 2
    const double *params;                  // kind 2: [ncurve][7]
    const int64_t *offsets;                // kind 2: [ncurve + 1]
    int64_t ncurve;
    int64_t stride;                        // work item i is input position i * stride (calibration
                                           // sub-samples use stride > 1; outputs stay compact)
    const double *ps, *pq, *prho;          // kind 3: per-position lens and source radius, with y1, y2
    const int32_t *list;                   // kind 3: optional list of positions; work item i is
                                           // position list[i] and its outputs go to index list[i]
};

struct KParams {
    WorkSrc src;
    double *out, *err;
    int32_t *nsamp;
    int8_t *pstat;
    char *arena;
    size_t slot_bytes;
    int cap;
    double tol;
    int chunk;                    // consecutive work items taken per atomic grab
    unsigned long long *counter;  // [0]: next work item; [1..5]: samples, FP64 sweeps, FP32 sweeps, edges,
                                  // FP64 Newton passes; [6]: queued repairs; [7]: next repair item
    int64_t *relist;              // work items queued for the repair pass (or null: no repairs)
    unsigned long long relist_cap;
    double *ld;                   // ld_kernel: per-warp node scratch (LD_WARP_DOUBLES per warp)
};

struct PosIn {
    double s, q, rho, y1, y2;
};

__device__ __forceinline__ bool pos_ok(double v) { return isfinite(v); }

// Straight-line trajectory (convention of twinkle.h).
__device__ __forceinline__ void trajectory(double u0, double alpha, double t0, double tE, double t, double &y1,
                                           double &y2) {
    const double tau = (t - t0) * rcp(tE);
    double sa, ca;
    sincos(alpha, &sa, &ca);
    y1 = tau * ca - u0 * sa;
    y2 = tau * sa + u0 * ca;
}

__device__ __forceinline__ bool fetch_position(const WorkSrc &w, int64_t idx, PosIn &P) {
    if (w.kind == 0 || w.kind == 5) {
        P.s = w.s; P.q = w.q; P.rho = w.rho;
        P.y1 = w.y1[idx];
        P.y2 = w.y2[idx];
    } else if (w.kind == 1) {
        P.s = w.s; P.q = w.q; P.rho = w.rho;
        trajectory(w.u0, w.alpha, w.t0, w.tE, w.times[idx], P.y1, P.y2);
    } else if (w.kind == 4) {
        // the binary's separation and axis angle change linearly with time
        const double dt = w.times[idx] - w.t0;
        P.s = w.s + w.ds_dt * dt; P.q = w.q; P.rho = w.rho;
        trajectory(w.u0, w.alpha + w.dalpha_dt * dt, w.t0, w.tE, w.times[idx], P.y1, P.y2);
    } else if (w.kind == 3) {
        const int64_t j = w.list ? (int64_t)w.list[idx] : idx;
        P.s = w.ps[j]; P.q = w.pq[j]; P.rho = w.prho[j];
        P.y1 = w.y1[j];
        P.y2 = w.y2[j];
    } else {
        // curve k with offsets[k] <= idx < offsets[k+1]
        int64_t lo = 0, hi = w.ncurve - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (w.offsets[mid] <= idx) lo = mid; else hi = mid - 1;
        }
        const double *pr = w.params + 7 * lo;
        P.s = pr[0]; P.q = pr[1]; P.rho = pr[2];
        const double tE = pr[6];
        if (!(tE > 0.0) || !isfinite(tE)) return false;
        trajectory(pr[3], pr[4], pr[5], tE, w.times[idx], P.y1, P.y2);
    }
    return P.s > 0.0 && P.q > 0.0 && P.rho > 0.0 && isfinite(P.s) && isfinite(P.q) && isfinite(P.rho) &&
           pos_ok(P.y1) && pos_ok(P.y2);
}

// REPAIR = false: the main pass over src.n work items.  REPAIR = true: the
// repair pass over the work items that the main pass queued in kp.relist
// (crossings that failed the slope test), integrated again with repairs.
// W = 1, 2 or 4 warps integrate each position together (the group's first
// warp takes the work items and writes the outputs; the group uses one arena
// slot and one shared-memory stage).
template <int PREC, int SPL, bool REPAIR, int OCC = TW_MIN_CTAS_PER_SM, int W = 1>
__global__ void __launch_bounds__(TPB, OCC) contour_kernel(KParams kp) {
    static_assert(WPB == CTA_WARPS, "CTA shape");
    __shared__ WarpStage stage[WPB];
    __shared__ Exch exch[WPB];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = wib / W;
    Coop<W> co;
    co.ex = &exch[grp * W];
    co.wig = wib % W;
    co.bar = 1 + grp;
    const int gw = blockIdx.x * (WPB / W) + grp;  // the group's arena slot
    const bool leader = co.wig == 0 && lane == 0;
    const Arena ar = arena_at(kp.arena, kp.slot_bytes, kp.cap, gw);
    unsigned long long n = (unsigned long long)kp.src.n;
    if (REPAIR) n = min(*(volatile unsigned long long *)(kp.counter + 6), kp.relist_cap);
    unsigned long long it = 0, end = 0, idx = 0;
    for (;;) {
        if (it >= end) {
            unsigned long long first = 0;
            if (leader) first = atomicAdd(kp.counter + (REPAIR ? 7 : 0), (unsigned long long)kp.chunk);
            if (W > 1) {
                if (leader) co.ex[0].first = first;
                co.sync();
                first = co.ex[0].first;
                co.sync();
            } else {
                first = __shfl_sync(FULL, first, 0);
            }
            it = first;
            end = it + (unsigned long long)kp.chunk;
            if (end > n) end = n;
            if (it >= end) break;
        }
        idx = REPAIR ? (unsigned long long)kp.relist[it] : it;
        PosIn P;
        const bool valid = fetch_position(kp.src, (int64_t)idx * kp.src.stride, P);
        double mu = __longlong_as_double(0x7ff8000000000000ll), err = mu;
        int nsamp = 0, status = PS_NONFINITE;
        if (valid) {
            // Swapping the masses (q -> 1/q) reflects the lens through the centre
            // of mass (Eq. 2), so mu(s, q, y1, y2) = mu(s, 1/q, -y1, y2).  Using it
            // for q > 1 keeps the lighter body in the role of the low-mass lens of
            // the refactored coefficients (Eq. 6).
            double q = P.q, y1 = P.y1;
            if (q > 1.0) { q = 1.0 / q; y1 = -y1; }
            LensK L;
            L.s = P.s;
            L.m1 = rcp(1.0 + q);
            L.m2 = q * L.m1;
            L.rho = P.rho;
            L.y0 = {y1 - P.s * L.m1, P.y2};  // centre-of-mass -> secondary frame
            // the 4-CTA instance serves per-position lenses: its root solver
            // keeps the pair loop rolled as well (see aberth_sweep)
            const PosResult r =
                integrate_position<PREC, SPL, REPAIR, (OCC >= 4), W>(L, kp.tol, kp.cap, ar, stage[grp * W], co);
            // a crossing failed the slope test: queue the position for the
            // repair pass (its outputs below are overwritten there)
            if (!REPAIR && (r.status & PS_SLOPE) && kp.relist && leader) {
                const unsigned long long k = atomicAdd(kp.counter + 6, 1ull);
                if (k < kp.relist_cap) kp.relist[k] = (int64_t)idx;
            }
            const double inv_src = rcp(3.141592653589793238 * P.rho * P.rho);
            mu = r.area * inv_src;
            err = r.err * inv_src;
            nsamp = r.nsamp;
            status = r.status;
            if (lane == 0) {  // every warp adds its own work; the sample count once
                if (co.wig == 0) atomicAdd(kp.counter + 1, (unsigned long long)r.nsamp);
                atomicAdd(kp.counter + 2, (unsigned long long)r.work.sw64);
                atomicAdd(kp.counter + 3, (unsigned long long)r.work.sw32);
                atomicAdd(kp.counter + 4, (unsigned long long)r.work.edges);
                atomicAdd(kp.counter + 5, (unsigned long long)r.work.nw64);
            }
            if (!isfinite(mu)) { status |= PS_NONFINITE; mu = __longlong_as_double(0x7ff8000000000000ll); }
        }
        if (leader) {
            const unsigned long long o = (kp.src.kind == 3 && kp.src.list) ? (unsigned long long)kp.src.list[idx] : idx;
            kp.out[o] = mu;
            if (kp.err) kp.err[o] = err;
            if (kp.nsamp) kp.nsamp[o] = nsamp;
            if (kp.pstat) kp.pstat[o] = (int8_t)status;
        }
        it++;
    }
}


// ---------------------------------------------------------- limb darkening
// A source of linear limb darkening I(r) = 1 - u (1 - sqrt(1 - r^2/rho^2))
// (the paper notes that contour integration of limb-darkened sources is
// costly, Sec. 1, and gives no method).  Integrating the image flux by parts
// over the radius, with r = rho sin(phi),
//   mu_LD = [(1 - u) mu(rho) + u Int_0^{pi/2} h(phi) dphi] / (1 - u/3),
//   h(phi) = sin^3(phi) mu(rho sin phi),
// mu(r) being the magnification of a uniform disc of radius r (the contour
// integral of integrate_position).  h has kinks where the circle of radius r
// touches the caustic, so the phi integral is adaptive Simpson: panels of
// five equally spaced nodes, four of width pi/8 to start (16 radii; h(0) =
// 0), each valued by the two half-panel Simpson rules with the Richardson
// correction, its error |S(panel) - S(halves)| / 15; a panel above its share
// of half the tolerance is split in two (four new radii), up to LD_MAXP
// panels.  Each uniform disc is integrated to the other half of the
// tolerance.  One warp per source; the panels live in a per-warp global
// scratch managed by lane 0.
constexpr int LD_MAXP = 24;       // panels
constexpr int LD_PSTRIDE = 7;     // a, w, h[5] per panel
constexpr int LD_SPLIT = 4;       // panel splits per round
constexpr int LD_WARP_DOUBLES = LD_MAXP * LD_PSTRIDE + 2 * LD_MAXP + 8 * LD_SPLIT;

template <int PREC>
__global__ void __launch_bounds__(TPB, TW_MIN_CTAS_PER_SM) ld_kernel(KParams kp) {
    __shared__ WarpStage stage[WPB];
    __shared__ Exch exch[WPB];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Coop<1> co;
    co.ex = &exch[wib];
    co.wig = 0;
    co.bar = 0;
    const int gw = blockIdx.x * WPB + wib;
    const Arena ar = arena_at(kp.arena, kp.slot_bytes, kp.cap, gw);
    double *pn = kp.ld + (size_t)gw * LD_WARP_DOUBLES;  // panels: a, w, h[0..4]
    double *pe = pn + LD_MAXP * LD_PSTRIDE;             // per panel: propagated disc error, Simpson error
    double *sp = pe + 2 * LD_MAXP;                      // this round's new nodes: angle, h, disc error, target
    const double halfpi = 1.5707963267948966192, u = kp.src.ld_u;
    const double tol_u = 0.5 * kp.tol;  // each uniform disc; the other half for the phi integral
    unsigned long long it = 0;
    for (;;) {
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(kp.counter, 1ull);
        it = __shfl_sync(FULL, first, 0);
        if (it >= (unsigned long long)kp.src.n) break;
        PosIn P;
        const bool valid = fetch_position(kp.src, (int64_t)it * kp.src.stride, P);
        double mu = __longlong_as_double(0x7ff8000000000000ll), err = mu;
        int nsamp = 0, status = PS_NONFINITE;
        if (valid) {
            double q = P.q, y1 = P.y1;
            if (q > 1.0) { q = 1.0 / q; y1 = -y1; }  // mass-swap symmetry (see contour_kernel)
            LensK L;
            L.s = P.s;
            L.m1 = rcp(1.0 + q);
            L.m2 = q * L.m1;
            L.y0 = {y1 - P.s * L.m1, P.y2};
            status = 0;
            WorkCount tw;
            // h at angle phi: a uniform disc of radius rho sin(phi)
            auto eval = [&](double phi, double &h, double &e) {
                const double sn = sin(phi);
                LensK Lr = L;
                Lr.rho = P.rho * sn;
                const PosResult r = integrate_position<PREC, 2, false, false, 1>(Lr, tol_u, kp.cap, ar, stage[wib], co);
                const double w3 = sn * sn * sn * rcp(3.141592653589793238 * Lr.rho * Lr.rho);
                h = w3 * r.area;
                e = w3 * r.err;
                status |= r.status;
                nsamp += r.nsamp;
                tw.sw64 += r.work.sw64;
                tw.sw32 += r.work.sw32;
                tw.edges += r.work.edges;
                tw.nw64 += r.work.nw64;
            };
            // four panels of width pi/8: nodes j pi/32, j = 1..16
            int np = 4;
            if (lane == 0)
                for (int p = 0; p < 4; p++) {
                    pn[p * LD_PSTRIDE] = p * halfpi / 4;
                    pn[p * LD_PSTRIDE + 1] = halfpi / 4;
                    pe[2 * p] = 0.0;
                }
            if (lane == 0) pn[2] = 0.0;  // h(0) = 0
            __syncwarp();
            for (int j = 1; j <= 16; j++) {
                double h, e;
                eval(halfpi * j / 16, h, e);
                if (lane == 0) {
                    const int p = (j - 1) / 4, k = (j - 1) % 4 + 1;  // node k of panel p
                    pn[p * LD_PSTRIDE + 2 + k] = h;
                    pe[2 * p] += 0.25 * e;
                    if (k == 4 && p + 1 < 4) pn[(p + 1) * LD_PSTRIDE + 2] = h;
                }
            }
            double T = 0.0, Eq = 0.0, Eu = 0.0;
            for (;;) {
                __syncwarp();
                int nsplit = 0;
                if (lane == 0) {
                    T = 0.0;
                    Eq = 0.0;
                    Eu = 0.0;
                    for (int p = 0; p < np; p++) {
                        const double *g = pn + p * LD_PSTRIDE;
                        const double w = g[1], *h = g + 2;
                        const double s1 = w / 6.0 * (h[0] + 4.0 * h[2] + h[4]);
                        const double s2 = w / 12.0 * (h[0] + 4.0 * h[1] + 2.0 * h[2] + 4.0 * h[3] + h[4]);
                        const double e = fabs(s2 - s1) / 15.0;
                        pe[2 * p + 1] = e;
                        T += s2 + (s2 - s1) / 15.0;
                        Eq += e;
                        Eu += w * pe[2 * p];
                    }
                    const double target = 0.5 * kp.tol * fabs(T);
                    if (Eq > target) {
                        while (nsplit < LD_SPLIT && np + nsplit < LD_MAXP) {
                            int pb = -1;
                            double eb = target / np;
                            for (int p = 0; p < np; p++)
                                if (pe[2 * p + 1] > eb && pn[p * LD_PSTRIDE + 1] > halfpi * 1e-6) {
                                    eb = pe[2 * p + 1];
                                    pb = p;
                                }
                            if (pb < 0) break;
                            pe[2 * pb + 1] = -1.0;  // taken
                            const double a = pn[pb * LD_PSTRIDE], w = pn[pb * LD_PSTRIDE + 1];
                            // the four new nodes of its halves, and which panel they split
                            for (int k = 0; k < 4; k++) sp[8 * nsplit + 2 * k] = a + w * (2 * k + 1) / 8.0;
                            sp[8 * nsplit + 1] = (double)pb;
                            nsplit++;
                        }
                    }
                }
                nsplit = __shfl_sync(FULL, nsplit, 0);
                __syncwarp();
                if (nsplit == 0) break;
                for (int j = 0; j < nsplit; j++) {
                    double hn[4], en[4];
                    for (int k = 0; k < 4; k++) eval(sp[8 * j + 2 * k], hn[k], en[k]);
                    if (lane == 0) {  // panel pb -> its left half in place, its right half appended
                        const int pb = (int)sp[8 * j + 1];
                        double *g = pn + pb * LD_PSTRIDE, *r = pn + np * LD_PSTRIDE;
                        const double a = g[0], w = g[1], h0 = g[2], h1 = g[3], h2 = g[4], h3 = g[5], h4 = g[6];
                        r[0] = a + 0.5 * w; r[1] = 0.5 * w;
                        r[2] = h2; r[3] = hn[2]; r[4] = h3; r[5] = hn[3]; r[6] = h4;
                        g[1] = 0.5 * w;
                        g[2] = h0; g[3] = hn[0]; g[4] = h1; g[5] = hn[1]; g[6] = h2;
                        const double eo = pe[2 * pb];
                        pe[2 * pb] = 0.5 * eo + 0.25 * (en[0] + en[1]);
                        pe[2 * np] = 0.5 * eo + 0.25 * (en[2] + en[3]);
                    }
                    np++;
                    __syncwarp();
                }
            }
            T = __shfl_sync(FULL, T, 0);
            Eq = __shfl_sync(FULL, Eq, 0);
            Eu = __shfl_sync(FULL, Eu, 0);
            // mu(rho): the node at pi/2, the last node of the panel that ends there
            double mrho = 0.0;
            if (lane == 0)
                for (int p = 0; p < np; p++)
                    if (fabs(pn[p * LD_PSTRIDE] + pn[p * LD_PSTRIDE + 1] - halfpi) < 1e-12) mrho = pn[p * LD_PSTRIDE + 6];
            mrho = __shfl_sync(FULL, mrho, 0);
            const double inv = 1.0 / (1.0 - u / 3.0);
            mu = ((1.0 - u) * mrho + u * T) * inv;
            err = ((1.0 - u) * tol_u * mrho + u * (Eu + Eq)) * inv;
            if (lane == 0) {
                atomicAdd(kp.counter + 1, (unsigned long long)nsamp);
                atomicAdd(kp.counter + 2, (unsigned long long)tw.sw64);
                atomicAdd(kp.counter + 3, (unsigned long long)tw.sw32);
                atomicAdd(kp.counter + 4, (unsigned long long)tw.edges);
                atomicAdd(kp.counter + 5, (unsigned long long)tw.nw64);
            }
            if (!isfinite(mu)) { status |= PS_NONFINITE; mu = __longlong_as_double(0x7ff8000000000000ll); }
        }
        if (lane == 0) {
            kp.out[it] = mu;
            if (kp.err) kp.err[it] = err;
            if (kp.nsamp) kp.nsamp[it] = nsamp;
            if (kp.pstat) kp.pstat[it] = (int8_t)status;
        }
    }
}

#define TW_DEFINE_LD_LAUNCHER(PREC)                                                                \
    cudaError_t launch_ld_##PREC(unsigned blocks, cudaStream_t st, const KParams &kp) {           \
        ld_kernel<PREC><<<blocks, TPB, 0, st>>>(kp);                                               \
        return cudaGetLastError();                                                                 \
    }                                                                                              \
    cudaError_t occupancy_ld_##PREC(int *occ) {                                                    \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, ld_kernel<PREC>, TPB, 0);        \
    }

// Host launcher and occupancy query of one kernel instance.
#define TW_DEFINE_LAUNCHER(PREC, SPL)                                                              \
    cudaError_t launch_contour_##PREC##_##SPL(unsigned blocks, cudaStream_t st, const KParams &kp) { \
        contour_kernel<PREC, SPL, false><<<blocks, TPB, 0, st>>>(kp);                               \
        return cudaGetLastError();                                                                  \
    }                                                                                               \
    cudaError_t occupancy_contour_##PREC##_##SPL(int *occ) {                                        \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, contour_kernel<PREC, SPL, false>, TPB, 0); \
    }

// An instance compiled for OCC CTAs per SM (a register budget of 65536 /
// (128 OCC) per thread): more resident warps hide more latency on positions
// whose warps diverge most (many lenses near caustics), at the price of
// register spills.
#define TW_DEFINE_LAUNCHER_OCC(PREC, SPL, OCC)                                                     \
    cudaError_t launch_contour_##PREC##_##SPL##_o##OCC(unsigned blocks, cudaStream_t st, const KParams &kp) { \
        contour_kernel<PREC, SPL, false, OCC><<<blocks, TPB, 0, st>>>(kp);                         \
        return cudaGetLastError();                                                                 \
    }                                                                                              \
    cudaError_t occupancy_contour_##PREC##_##SPL##_o##OCC(int *occ) {                              \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, contour_kernel<PREC, SPL, false, OCC>, TPB, 0); \
    }

// An instance in which W warps integrate each position (one sample per lane).
#define TW_DEFINE_LAUNCHER_W(PREC, W)                                                              \
    cudaError_t launch_contour_##PREC##_w##W(unsigned blocks, cudaStream_t st, const KParams &kp) { \
        contour_kernel<PREC, 1, false, TW_MIN_CTAS_PER_SM, W><<<blocks, TPB, 0, st>>>(kp);          \
        return cudaGetLastError();                                                                  \
    }                                                                                               \
    cudaError_t occupancy_contour_##PREC##_w##W(int *occ) {                                         \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, contour_kernel<PREC, 1, false, TW_MIN_CTAS_PER_SM, W>, \
                                                             TPB, 0);                               \
    }

// The repair-pass instance of a precision (two samples per lane).
#define TW_DEFINE_REPAIR_LAUNCHER(PREC)                                                            \
    cudaError_t launch_repair_##PREC(unsigned blocks, cudaStream_t st, const KParams &kp) {       \
        contour_kernel<PREC, 2, true><<<blocks, TPB, 0, st>>>(kp);                                 \
        return cudaGetLastError();                                                                 \
    }

#define TW_DECLARE_LAUNCHER(PREC, SPL)                                                           \
    cudaError_t launch_contour_##PREC##_##SPL(unsigned blocks, cudaStream_t st, const KParams &kp); \
    cudaError_t occupancy_contour_##PREC##_##SPL(int *occ);

cudaError_t launch_rcp_selftest(unsigned long long *max_err_bits, int n, cudaStream_t st);
// FMA throughput probe (k_selftest.cu): kind 0 FP64, 1 FP32; returns 0 or -1.
int fma_probe(int kind, int nsm, double *flops_per_s);

// Host (twinkle.cu): contour integration of n positions with per-position lens
// and source radius (kind 3), device pointers, serialised with the library's
// other launches.  With `list`, work item i is position list[i] and writes
// out[list[i]] (and status[list[i]]).  Returns a TW_* code.
int contour_positions(const double *s, const double *q, const double *rho, const double *y1, const double *y2,
                      const int32_t *list, int64_t n, double tol, int prec, int max_samples, double *out,
                      int8_t *status, cudaStream_t st);

TW_DECLARE_LAUNCHER(0, 1)
TW_DECLARE_LAUNCHER(0, 2)
TW_DECLARE_LAUNCHER(0, 4)
TW_DECLARE_LAUNCHER(1, 1)
TW_DECLARE_LAUNCHER(1, 2)
TW_DECLARE_LAUNCHER(1, 4)
cudaError_t launch_contour_0_2_o4(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_0_2_o4(int *occ);
cudaError_t launch_contour_1_2_o4(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_1_2_o4(int *occ);
cudaError_t launch_contour_0_w2(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_0_w2(int *occ);
cudaError_t launch_contour_1_w2(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_1_w2(int *occ);
cudaError_t launch_contour_0_w4(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_0_w4(int *occ);
cudaError_t launch_contour_1_w4(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_1_w4(int *occ);
cudaError_t launch_ld_0(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_ld_0(int *occ);
cudaError_t launch_ld_1(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_ld_1(int *occ);
cudaError_t launch_repair_0(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t launch_repair_1(unsigned blocks, cudaStream_t st, const KParams &kp);

}  // namespace tw
