// contour.cuh -- contour integration of one source position by one warp.
//
// The limb is sampled at angles theta (Sec. 2.3: counter-clockwise from +x,
// the sort key of the samples).  Each sample holds its five roots, which of
// them are real images and with which parity, and dz/dtheta and z' ^ z'' of
// each (lens.cuh).  Each edge between consecutive samples contributes
//   - for every pair of same-parity images linked across it (Sec. 2.3: same
//     parity, minimum total distance), p * [trapezium (Eq. 9) + parabolic
//     correction (Eq. 10, mean of the two forms)], and the error terms
//     E1..E4 of Eq. 17;
//   - where the image count changes (a caustic crossing, Sec. 2.3), the extra
//     positive/negative pair of the five-image sample is joined to itself by
//     the cross-caustic correction of Eq. 11 with the errors of Eq. 18.
// The area is the sum over edges (Eq. 8); sampling stops once the summed
// error is at most rel_tol * area (Sec. 2.5, Sec. 3).  Otherwise new angles
// are drawn by inverse-transform sampling of the cumulative per-edge error,
// with each edge's share of the tolerance subtracted first, at
// (j + 1/2)/n_new quantiles (Sec. 2.5), merged into the sorted order, and only
// the edges touching new samples are recomputed (Sec. 3).
//
// Lane layout: a warp owns one position; the initial 32*SPL uniform samples
// and every batch of 32*SPL new samples are spread SPL per lane; sums and the
// cumulative error use warp shuffles.  Per-sample records live in the warp's
// slot of a global arena (structure of arrays, L2-resident in practice);
// only the current batch of new angles is staged in shared memory.
#pragma once
#include <stdint.h>

#include "lens.cuh"

namespace tw {

constexpr unsigned FULL = 0xffffffffu;

// Position status bits (mirrors TW_POS_* of twinkle.h).
enum : int { PS_CAP = 1, PS_IMAGECOUNT = 2, PS_NONFINITE = 4, PS_SOLVER = 8, PS_SLOPE = 16 };
// Returned by compute_edge for an edge across a caustic (internal; never in a status).
constexpr int EDGE_XING = 64;
// A limb that crosses a caustic stops at this fraction of the tolerance: on
// crossing limbs sampled by a few batches the error estimate of Eq. 18 was
// measured below the true error by up to 1.4x (paper's Fig. 4 grid at s = 0.5,
// rho = 5e-5), never on limbs without crossings.
constexpr double XING_TOL_FACTOR = 0.5;

// One warp slot of the sample arena.  Records are indexed by sample slot (the
// order in which samples were created); ordA/ordB hold slot numbers in theta
// order; eA/eE the edge from a slot to its successor in theta order.
struct Arena {
    double *theta;
    cxd *roots;  // [slot*5 + i]
    cxf *zp;     // [slot*5 + i]
    float *w;    // [slot*5 + i]
    uint32_t *meta;
    double *eA;
    double *eE;
    uint16_t *ordA;
    uint16_t *ordB;
    double *cum;
};

__host__ __device__ constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of one warp slot for a sample cap `cap`.
__host__ __device__ constexpr size_t arena_slot_bytes(int cap) {
    const size_t c = (size_t)cap;
    return align256(c * 8) + align256(c * 5 * 16) + align256(c * 5 * 8) + align256(c * 5 * 4) + align256(c * 4) +
           align256(c * 8) * 2 + align256(c * 2) * 2 + align256(c * 8);
}

__device__ inline Arena arena_at(char *base, size_t slot_bytes, int cap, int slot) {
    char *p = base + slot_bytes * (size_t)slot;
    const size_t c = (size_t)cap;
    Arena a;
    a.theta = (double *)p; p += align256(c * 8);
    a.roots = (cxd *)p; p += align256(c * 5 * 16);
    a.zp = (cxf *)p; p += align256(c * 5 * 8);
    a.w = (float *)p; p += align256(c * 5 * 4);
    a.meta = (uint32_t *)p; p += align256(c * 4);
    a.eA = (double *)p; p += align256(c * 8);
    a.eE = (double *)p; p += align256(c * 8);
    a.ordA = (uint16_t *)p; p += align256(c * 2);
    a.ordB = (uint16_t *)p; p += align256(c * 2);
    a.cum = (double *)p;
    return a;
}

struct Img {
    cxd z;   // image position (FP64: the trapezium terms need it)
    cxf zp;  // dz/dtheta
    float w; // z' ^ z''
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Normal link of image a (angle theta) to image b (theta + dth) of parity sgn:
// trapezium (Eq. 9, FP64) plus the mean of the two parabolic corrections
// (Eq. 10), and the error terms E1..E4 of Eq. 17 (FP32: corrections are many
// orders below the area and only need relative accuracy).
__device__ __forceinline__ void link_contrib(const Img &a, const Img &b, double sgn, float dth, double &dA,
                                             float &dE) {
    const float d2 = dth * dth, d3 = d2 * dth;
    const double At = 0.5 * wedge(a.z, b.z);
    const float p1 = (a.w + b.w) * d3 * (1.0f / 24.0f);
    const cxf dz = to_f(b.z - a.z), dzp = b.zp - a.zp;
    const float p2 = wedge(dz, dzp) * dth * (1.0f / 12.0f);
    const float Ap = 0.5f * (p1 + p2);
    dA += sgn * (At + (double)Ap);
    const float e1 = fabsf(a.w - b.w) * d3 * (1.0f / 48.0f);
    const float dt = fabsf(dot(a.zp, b.zp));
    const float e2 = 1.5f * fabsf(Ap * (norm2(dz) / fmaxf(d2 * dt, 1e-37f) - 1.0f));
    const float e3 = 0.1f * fabsf(Ap) * d2;
    const float e4 = fabsf(p1 - p2);
    dE += e1 + e2 + e3 + e4;
}

// Extra positive (P) / negative (M) pair of a five-image sample next to a
// caustic crossing, joined to itself: chord from the incoming to the outgoing
// track (M -> P when the pair is created towards +theta, P -> M when it is
// destroyed) plus the cross-caustic correction of Eq. 11 and its errors
// (Eq. 18; the sign inside E2 is - for a creation).  dth is the edge's step.
__device__ __forceinline__ void pair_contrib(const Img &P, const Img &M, bool creation, float dth, double &dA,
                                             float &dE) {
    const cxf dz = to_f(P.z - M.z);
    const float adz = sqrtf(norm2(dz));
    const float dt = fabsf(dot(P.zp, M.zp));
    float tt = (dt > 0.0f) ? adz * rsqrtf(dt) : 4.0f * dth;  // Eq. 11: |z+ - z-| / sqrt|z'+ . z'-|
    tt = fminf(tt, 4.0f * dth);
    const float t3 = tt * tt * tt;
    const float Ap = (P.w - M.w) * t3 * (1.0f / 24.0f);
    const double At = creation ? 0.5 * wedge(M.z, P.z) : 0.5 * wedge(P.z, M.z);
    dA += At + (double)Ap;
    const float e1 = fabsf(P.w + M.w) * t3 * (1.0f / 48.0f);
    const cxf dzp = P.zp - M.zp;
    const float proj = dot(dz, dzp);
    const float sq = 2.0f * adz * sqrtf(dt);
    const float e2 = 1.5f * fabsf(creation ? proj - sq : proj + sq) * tt;
    const float e3 = 0.1f * fabsf(Ap) * dth * dth;
    dE += e1 + e2 + e3;
}

// i-th entry of the p-th permutation of N <= 3 elements.
template <int N>
__device__ __forceinline__ constexpr int perm_at(int p, int i) {
    return N == 1 ? 0
         : N == 2 ? (p == 0 ? i : 1 - i)
         : (p == 0 ? (i == 0 ? 0 : i == 1 ? 1 : 2)
          : p == 1 ? (i == 0 ? 0 : i == 1 ? 2 : 1)
          : p == 2 ? (i == 0 ? 1 : i == 1 ? 0 : 2)
          : p == 3 ? (i == 0 ? 1 : i == 1 ? 2 : 0)
          : p == 4 ? (i == 0 ? 2 : i == 1 ? 0 : 1)
          :          (i == 0 ? 2 : i == 1 ? 1 : 0));
}

// Link the NX images of one parity class at the edge's start (positions X,
// class slots x0..x0+NX-1) to the NY images of that class at its end (Y,
// y0..), |NX - NY| <= 1, so that the total distance is minimal (Sec. 2.3;
// ties go to the lowest permutation).  Appends each link as a 3-bit start
// slot, a 3-bit end slot and a parity bit to `links`; returns the slot of the
// image left over when NX != NY (else -1).
template <int NX, int NY>
__device__ __forceinline__ int link_class(const cxd *X, const cxd *Y, int x0, int y0, unsigned neg, uint64_t &links,
                                          int &nlinks) {
    constexpr int N = NX > NY ? NX : NY;
    constexpr int M = NX > NY ? NY : NX;
    constexpr int NP = N == 1 ? 1 : (N == 2 ? 2 : 6);
    // each distance once (the permutations share them)
    float dist[NX][NY];
#pragma unroll
    for (int a = 0; a < NX; a++)
#pragma unroll
        for (int b = 0; b < NY; b++) dist[a][b] = sqrtf(norm2(to_f(Y[y0 + b] - X[x0 + a])));
    float best_cost = 3.0e38f;
    int best = 0;
#pragma unroll
    for (int p = 0; p < NP; p++) {
        float cost = 0.f;
#pragma unroll
        for (int i = 0; i < M; i++) {
            const int j = perm_at<N>(p, i);
            cost += (NX <= NY) ? dist[i][j] : dist[j][i];
        }
        if (cost < best_cost) { best_cost = cost; best = p; }
    }
    int left = -1;
#pragma unroll
    for (int p = 0; p < NP; p++) {
        if (p == best) {
#pragma unroll
            for (int i = 0; i < M; i++) {
                const int j = perm_at<N>(p, i);
                const unsigned a = (unsigned)(NX <= NY ? x0 + i : x0 + j), b = (unsigned)(NX <= NY ? y0 + j : y0 + i);
                links |= (uint64_t)(a | (b << 3) | (neg << 6)) << (7 * nlinks);
                nlinks++;
            }
            if (NX < NY) left = y0 + perm_at<N>(p, N - 1);
            if (NX > NY) left = x0 + perm_at<N>(p, N - 1);
        }
    }
    return left;
}

// Linking of one edge given the image positions of its two samples (class
// slots in parity order, positives first).  lp/ln: slots of the extra
// positive/negative image when the count changes.
template <int NA, int NB>
__device__ __forceinline__ void edge_links(const cxd *ZA, const cxd *ZB, uint64_t &links, int &nlinks, int &lp, int &ln) {
    constexpr int PA = (NA - 1) / 2, PB = (NB - 1) / 2;
    lp = link_class<PA, PB>(ZA, ZB, 0, 0, 0u, links, nlinks);
    ln = link_class<NA - PA, NB - PB>(ZA, ZB, PA, PB, 1u, links, nlinks);
}

__device__ __forceinline__ Img load_img(const Arena &ar, int slot, uint32_t meta, int k) {
    const int i = slot * 5 + meta_index(meta, k);
    Img m;
    m.z = ar.roots[i];
    m.zp = ar.zp[i];
    m.w = ar.w[i];
    return m;
}

__device__ __forceinline__ unsigned real_mask(uint32_t meta) {
    unsigned m = 0;
    const int n = meta_count(meta);
    for (int k = 0; k < n; k++) m |= 1u << meta_index(meta, k);
    return m;
}

// Slope test (Sec. 2.4.2).  Near a critical curve the separation of the two
// images that merge there is the square root of a quantity that changes sign
// across the caustic, so the difference of the pair that is real on the
// five-image side and the difference of the ghost pair on the three-image
// side are perpendicular, while the differences of one pair at neighbouring
// samples of the same side are nearly parallel.  The local form holds only
// while both pairs are close compared with the other images.
//
// Relation of two pairs with differences d1, d2 whose midpoints lie at
// squared distances o1, o2 from the nearest other image: +1 both local
// (|d|^2 < o/16) and perpendicular (cos^2 < 1/4), -1 both local and parallel
// (cos^2 > 0.81), 0 otherwise.
__device__ __forceinline__ int pair_relation(cxf d1, float o1, cxf d2, float o2) {
    const float n1 = norm2(d1), n2 = norm2(d2);
    if (!(n1 < 0.0625f * o1 && n2 < 0.0625f * o2)) return 0;
    const float c = dot(d1, d2), c2 = c * c, nn = n1 * n2;
    return c2 < 0.25f * nn ? 1 : (c2 > 0.81f * nn ? -1 : 0);
}

// Pair (class slots kp, kn) of the five-image sample s5: difference P - M and
// squared distance from its midpoint to the nearest other real image.
__device__ __forceinline__ cxf pair5(const Arena &ar, int s5, uint32_t m5, int kp, int kn, float &o) {
    const cxf P = to_f(ar.roots[s5 * 5 + meta_index(m5, kp)]), M = to_f(ar.roots[s5 * 5 + meta_index(m5, kn)]);
    const cxf c = 0.5f * (P + M);
    o = 3.0e38f;
    for (int k = 0; k < 5; k++)
        if (k != kp && k != kn) o = fminf(o, norm2(to_f(ar.roots[s5 * 5 + meta_index(m5, k)]) - c));
    return P - M;
}

// Ghost pair of the three-image sample s3: difference and squared distance
// from its midpoint to the nearest real image.
__device__ __forceinline__ cxf ghost3(const Arena &ar, int s3, uint32_t m3, float &o) {
    const unsigned real3 = real_mask(m3);
    cxf G[2] = {{0.f, 0.f}, {0.f, 0.f}};
    int ng = 0;
    for (int i = 0; i < 5; i++)
        if (!((real3 >> i) & 1u) && ng < 2) G[ng++] = to_f(ar.roots[s3 * 5 + i]);
    const cxf c = 0.5f * (G[0] + G[1]);
    o = 3.0e38f;
    for (int k = 0; k < 3; k++) o = fminf(o, norm2(to_f(ar.roots[s3 * 5 + meta_index(m3, k)]) - c));
    return G[0] - G[1];
}

// Crossing at an edge: true when the extra pair of its five-image sample and
// the ghost pair of its three-image sample are parallel, i.e. the crossing is
// misplaced (a ghost pair was taken for real).
__device__ __forceinline__ bool slope_violation(const Arena &ar, int s5, uint32_t m5, int kp, int kn, int s3,
                                                uint32_t m3) {
    float o5, o3;
    const cxf d5 = pair5(ar, s5, m5, kp, kn, o5), d3 = ghost3(ar, s3, m3, o3);
    return pair_relation(d5, o5, d3, o3) == -1;
}

// Area and error of the edge from sample slot sa to slot sb (angle step dth).
// Returns PS_SLOPE when the edge is a caustic crossing that fails the slope
// test.
__device__ __forceinline__ void link_edge(const Arena &ar, int sa, int sb, uint32_t ma, uint32_t mb, uint64_t &links,
                                          int &nlinks, int &lp, int &ln) {
    const int na = meta_count(ma), nb = meta_count(mb);
    cxd ZA[5], ZB[5];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        if (k < na) ZA[k] = ar.roots[sa * 5 + meta_index(ma, k)];
        if (k < nb) ZB[k] = ar.roots[sb * 5 + meta_index(mb, k)];
    }
    links = 0;
    nlinks = 0;
    lp = ln = -1;
    if (na == 3 && nb == 3) edge_links<3, 3>(ZA, ZB, links, nlinks, lp, ln);
    else if (na == 5 && nb == 5) edge_links<5, 5>(ZA, ZB, links, nlinks, lp, ln);
    else if (na == 3) edge_links<3, 5>(ZA, ZB, links, nlinks, lp, ln);
    else edge_links<5, 3>(ZA, ZB, links, nlinks, lp, ln);
}

static __device__ __noinline__ int compute_edge(const Arena &ar, int sa, int sb, double dth, double *outA, double *outE,
                                                bool guard) {
    const uint32_t ma = ar.meta[sa], mb = ar.meta[sb];
    const int na = meta_count(ma), nb = meta_count(mb);
    uint64_t links;
    int nlinks, lp, ln, flags = 0;
    link_edge(ar, sa, sb, ma, mb, links, nlinks, lp, ln);
    double dA = 0.0;
    float dE = 0.0f;
    const float dthf = (float)dth;
    for (int k = 0; k < nlinks; k++) {
        const unsigned l = (unsigned)(links >> (7 * k)) & 127u;
        const Img a = load_img(ar, sa, ma, (int)(l & 7u)), b = load_img(ar, sb, mb, (int)((l >> 3) & 7u));
        link_contrib(a, b, (l >> 6) ? -1.0 : 1.0, dthf, dA, dE);
    }
    if (na != nb) {
        flags |= EDGE_XING;
        // the extra pair belongs to the five-image end of the edge
        const bool creation = na < nb;
        const int sl = creation ? sb : sa;
        const uint32_t ml = creation ? mb : ma;
        pair_contrib(load_img(ar, sl, ml, lp), load_img(ar, sl, ml, ln), creation, dthf, dA, dE);
        if (slope_violation(ar, sl, ml, lp, ln, creation ? sa : sb, creation ? ma : mb)) flags |= PS_SLOPE;
    }
    double dEd = (double)dE;
    // a sample that failed the image-count check: keep refining around it
    if ((ma | mb) >> 31) dEd += fabs(dA);
    // Two three-image samples with the caustic close to one of them: a pair
    // of crossings closer than the sample spacing (a five-image stretch no
    // sample has seen) would leave the error terms smooth and the area short
    // by that stretch.  A crossing inside the edge lies within half the edge
    // of the nearer sample, so that sample's distance to the caustic
    // (classify_store, in units of rho) is at most half the edge; its
    // estimate is within a factor 2 there (measured against the oracle's
    // caustic; a sample farther away, next to a cusp, was overestimated up
    // to 150x, so the smaller of the two is used).  The edge is refined like an image-count
    // failure while it is longer than half that smaller distance, until a
    // crossing is sampled or the caustic is shown to stay away.  Samples
    // re-judged by the slope repair carry no distance and are skipped.  The
    // caller turns the guard off once the limb shows a crossing: next to a
    // sampled crossing the outer edge would otherwise be refined again every
    // time the crossing edge is (the nearer sample's distance shrinking with
    // it), and the narrow dip it looks for is the case with no crossing seen.
    if (guard && na == 3 && nb == 3 && !((ma | mb) >> 30)) {
        const int ga = __ffs(~real_mask(ma) & 31u) - 1, gb = __ffs(~real_mask(mb) & 31u) - 1;
        if (dthf > 0.5f * fminf(ar.w[sa * 5 + ga], ar.w[sb * 5 + gb])) dEd += fabs(dA);
    }
    *outA = dA;
    *outE = dEd;
    return flags;
}

// Repair of a crossing that failed the slope test, at the edge from theta
// position p to p + 1 (ord: slots in theta order, N samples, cyclic), after
// Sec. 2.4.2: starting at the crossing's five-image sample, the extra pair is
// followed into the five-image run (at each sample the positive and negative
// images nearest to the previous pair's) until
//   - two consecutive pairs are perpendicular: the jump of the slope is there,
//     and the samples before it carried a ghost pair taken for real; they are
//     re-judged as three-image samples (the crossing moves to the jump);
//   - the run ends at a three-image sample whose crossing also fails the
//     test: the whole run is a false image piece and is re-judged.
// Otherwise (pairs no longer close, a failed sample, 64 samples walked)
// nothing is changed.  Re-judged samples carry meta bit 30 and are never
// re-judged again; the edges around them are recomputed.  Runs on one lane.
constexpr int SLOPE_WALK = 64;

static __device__ __noinline__ int slope_fix(const Arena &ar, const uint16_t *ord, int N, int p) {
    const double twopi = 6.283185307179586476925287;
    auto slot = [&](int i) { return (int)ord[((i % N) + N) % N]; };
    const int sa = slot(p), sb = slot(p + 1);
    const uint32_t ma = ar.meta[sa], mb = ar.meta[sb];
    if ((ma | mb) >> 30) return PS_SLOPE;
    const int na = meta_count(ma), nb = meta_count(mb);
    if (na == nb) return 0;
    uint64_t links;
    int nlinks, kp, kn;
    link_edge(ar, sa, sb, ma, mb, links, nlinks, kp, kn);
    const int dir = na == 5 ? -1 : 1;  // from the crossing into the five-image run
    const int first = na == 5 ? p : p + 1;
    uint8_t pk[SLOPE_WALK];  // pair (kp | kn << 3) of each walked sample
    int len = 0, j = first, s5 = slot(first);
    uint32_t m5 = ar.meta[s5];
    bool rejudge = false;
    for (;;) {
        pk[len++] = (uint8_t)(kp | (kn << 3));
        float o;
        const cxf d = pair5(ar, s5, m5, kp, kn, o);
        const cxf P = to_f(ar.roots[s5 * 5 + meta_index(m5, kp)]), M = to_f(ar.roots[s5 * 5 + meta_index(m5, kn)]);
        const int sn = slot(j + dir);
        const uint32_t mn = ar.meta[sn];
        if (mn >> 30) return PS_SLOPE;
        if (meta_count(mn) == 3) {
            // the far end of the run: a false piece when that crossing fails too
            float o3;
            const cxf d3 = ghost3(ar, sn, mn, o3);
            rejudge = pair_relation(d, o, d3, o3) == -1;
            break;
        }
        // the next sample's pair: positive image nearest P, negative nearest M
        int np = 0, nn = 2;
        float bp = 3.0e38f, bn = 3.0e38f;
        for (int k = 0; k < 5; k++) {
            const cxf z = to_f(ar.roots[sn * 5 + meta_index(mn, k)]);
            if (k < 2) { const float t = norm2(z - P); if (t < bp) { bp = t; np = k; } }
            else { const float t = norm2(z - M); if (t < bn) { bn = t; nn = k; } }
        }
        float on;
        const cxf dn = pair5(ar, sn, mn, np, nn, on);
        const int rel = pair_relation(d, o, dn, on);
        if (rel == 1) { rejudge = true; break; }  // the jump
        if (rel == 0 || len == SLOPE_WALK || len >= N - 2) break;
        j += dir;
        s5 = sn;
        m5 = mn;
        kp = np;
        kn = nn;
    }
    if (!rejudge) return PS_SLOPE;
    // re-judge the walked samples: drop their pair, keep the other three images
    for (int t = 0; t < len; t++) {
        const int sl = slot(first + dir * t);
        const uint32_t m = ar.meta[sl];
        const int a = pk[t] & 7, b = pk[t] >> 3;
        uint32_t nm = 3u | (1u << 30);
        int k3 = 0;
        for (int k = 0; k < 5; k++)
            if (k != a && k != b) { nm |= (uint32_t)meta_index(m, k) << (3 + 3 * k3); k3++; }
        ar.meta[sl] = nm;
    }
    // recompute the edges touching them
    const int lo = dir > 0 ? first - 1 : first - len;
    int flags = PS_SLOPE;
    for (int e = lo; e <= lo + len; e++) {
        const int ee = ((e % N) + N) % N;
        const int s0 = ord[ee], s1 = ord[(ee + 1) % N];
        const double t1 = (ee + 1 < N) ? ar.theta[s1] : ar.theta[s1] + twopi;
        compute_edge(ar, s0, s1, t1 - ar.theta[s0], &ar.eA[s0], &ar.eE[s0], false);
    }
    return flags;
}

// One limb sample: coefficients, roots (warm-started from z), classification,
// derivatives, stored in slot `slot`.  Returns the sample's status bits.
// Work done by one warp on one position (for FLOP accounting).
struct WorkCount {
    int sw64 = 0, sw32 = 0, edges = 0, nw64 = 0;
};

// First-order warm start: each real image (bit i of `mask`) is moved by dz_i
// when that step is small against its distance to the nearest other root
// (far from a critical curve, where the linear prediction holds).
__device__ __forceinline__ void predict_roots(cxd z[5], const cxf dz[5], unsigned mask) {
    cxf zf[5];
#pragma unroll
    for (int i = 0; i < 5; i++) zf[i] = to_f(z[i]);
#pragma unroll
    for (int i = 0; i < 5; i++) {
        if (!((mask >> i) & 1u)) continue;
        float sep2 = 3.0e38f;
#pragma unroll
        for (int j = 0; j < 5; j++)
            if (j != i) sep2 = fminf(sep2, norm2(zf[i] - zf[j]));
        if (norm2(dz[i]) < 0.04f * sep2) z[i] = z[i] + to_d(dz[i]);
    }
}

template <int PREC, bool RP = false>
static __device__ __noinline__ int limb_sample(const LensK &L, double th, cxd z[5], const Arena &ar, int slot,
                                               WorkCount &wc) {
    double sn, cs;
    sincos(th, &sn, &cs);
    const cxd y = {L.y0.x + L.rho * cs, L.y0.y + L.rho * sn};
    const cxd dzeta = {-L.rho * sn, L.rho * cs}; // zeta' = i rho e^{i theta}
    cxd c[6];
    eq6_coeffs(L.s, L.m2, y, c);
    if (!roots_finite(z)) initial_roots(L.s, y, z);
    float dpa[5], ca[6];
    int f = solve_quintic<PREC, RP>(c, z, dpa, 60, wc.sw64, wc.sw32, wc.nw64, ca);
    SampleRefs o = {&ar.theta[slot], &ar.roots[slot * 5], &ar.zp[slot * 5], &ar.w[slot * 5], &ar.meta[slot]};
    f |= classify_store(L, y, dzeta, ca, z, dpa, th, o);
    return f;
}

struct WarpStage {
    double theta_new[256];
    uint16_t pos_new[256];
};

struct PosResult {
    double area, err;
    int nsamp, status;
    WorkCount work;  // summed over the warp
};

// Repairs (one lane at a time) of the crossings that failed the slope test:
// vpos is this lane's edge position, or -1.  Returns status bits (the same on
// every lane).
static __device__ __noinline__ int slope_repairs(const Arena &ar, const uint16_t *ord, int N, int vpos) {
    const int lane = threadIdx.x & 31;
    unsigned vb = __ballot_sync(FULL, vpos >= 0);
    int f = 0;
    while (vb) {
        const int src = __ffs(vb) - 1;
        const int p = __shfl_sync(FULL, vpos, src);
        if (lane == 0) f |= slope_fix(ar, ord, N, p);
        __syncwarp();
        vb &= vb - 1;
    }
    return __shfl_sync(FULL, f, 0);
}

constexpr int CTA_WARPS = 4;  // warps per CTA of the contour kernels

// Cooperation of the W warps (1, 2 or 4 of a CTA's four) that integrate one
// position together: a barrier over the group, and one exchange slot per warp
// in shared memory for the group's sums, scans and compactions.  Every
// decision that ends a loop is taken from values read back from these slots
// after a barrier, so all warps of a group take it alike.
struct Exch {
    double a, e, scan, last_th;
    unsigned long long first;
    int cnt, last_pos, flags, xing;
};

template <int W>
struct Coop {
    Exch *ex;  // this group's W slots
    int wig;   // warp index in the group
    int bar;   // named barrier of the group (W = 2: 1 or 2, 64 threads each)
    __device__ __forceinline__ void sync() const {
        if (W == 1) __syncwarp();
        else if (W == CTA_WARPS) __syncthreads();
        else if (bar == 1) asm volatile("bar.sync 1, 64;" ::: "memory");
        else asm volatile("bar.sync 2, 64;" ::: "memory");
    }
};

// REPAIR = false: a crossing that fails the slope test only sets PS_SLOPE
// (the position is then integrated again by the REPAIR = true instance, which
// repairs such crossings as they appear; it runs four warps per position, so
// that the few, long repaired positions use every scheduler of an SM).
// Keeping the repair code out of the main instance keeps its register
// allocation unchanged.
// W warps share the position: 32 W SPL samples per iteration, lane gl = 32 wig
// + lane of the group taking samples gl SPL .. gl SPL + SPL - 1 of a batch.
// PosResult.work is this warp's own share.
template <int PREC, int SPL, bool REPAIR, bool RP = false, int W = 1>
__device__ PosResult integrate_position(const LensK &L, double tol, int cap, const Arena &ar, WarpStage &ws,
                                        const Coop<W> &co) {
    static_assert(W == 1 || W == 2 || W == CTA_WARPS, "1, 2 or 4 warps per position");
    static_assert(32 * SPL * W <= 256, "a batch must fit the shared-memory stage");
    constexpr int SPI = 32 * SPL * W;
    const int lane = threadIdx.x & 31;
    const int gl = co.wig * 32 + lane;
    const double twopi = 6.283185307179586476925287;
    const double minsep = 1e-15 / L.rho + 1e-14;
    int flags = 0;
    WorkCount wc;
    int vpos = -1;  // theta position of an edge that failed the slope test
    bool xe = false;  // this lane has computed an edge across a caustic

    // Images of a point inside the source: the warm start of the first samples.
    // The point is offset from the centre by rho/2 because Eq. 6 degenerates
    // (c5 = 0, a root at infinity) when the source point sits on a lens, and
    // source centres exactly on a lens are a common input.  This solve only
    // provides starting points (every sample is then iterated to full FP64
    // accuracy in either mode), so it runs in FP32 from a cold start; it is
    // the same on every lane (and every warp of a group).
    const cxd yw = {L.y0.x + 0.5 * L.rho * 0.7648421872844885, L.y0.y + 0.5 * L.rho * 0.6442176872376911};
    cxd zc[5];
    unsigned cmask = 0x1fu;  // real images of the warm-start point
    cxf cf1[5];              // f' at those images
    float crJ[5];            // 1/J at those images
    {
        cxd cc[6];
        eq6_coeffs(L.s, L.m2, yw, cc);
        float ca[6];
        abs_coeffs(cc, ca);
        const float cm = fmaxf(fmaxf(fmaxf(ca[0], ca[1]), fmaxf(ca[2], ca[3])), fmaxf(ca[4], ca[5]));
        const double sc = 1.0 / (double)cm;
        cxf cf[6];
        float caf[6];
#pragma unroll
        for (int k = 0; k < 6; k++) {
            cf[k] = to_f(sc * cc[k]);
            caf[k] = ca[k] / cm;
        }
        // cold start on a circle enclosing the roots
        const float r0 = 1.5f * (1.0f + (float)L.s + sqrtf((float)norm2(yw)));
        // unit vectors at angles 2 pi k/5 + 0.4
        const float ux[5] = {0.92106099f, -0.08573535f, -0.97404836f, -0.51625964f, 0.65498235f};
        const float uy[5] = {0.38941834f, 0.99631795f, 0.22634001f, -0.85643213f, -0.75564417f};
        cxf zf[5];
#pragma unroll
        for (int k = 0; k < 5; k++) zf[k] = {-0.5f * (float)L.s + r0 * ux[k], r0 * uy[k]};
        float dpa[5];
        int it = 0;
        for (; it < 100; it++)
            if (aberth_sweep<float>(cf, caf, zf, dpa, 2e-6f, 6e-8f)) break;
        if (lane == 0) wc.sw32 += it + 1;
        bool fin = true;
#pragma unroll
        for (int i = 0; i < 5; i++) {
            zc[i] = to_d(zf[i]);
            fin = fin && isfinite(zf[i].x) && isfinite(zf[i].y);
        }
        if (!fin) initial_roots(L.s, L.y0, zc);
        // real images by the residual pair test (Sec. 2.4.1), and the
        // first-order response dz = (dzeta - conj(f') conj(dzeta))/J of each
        // to a move dzeta of the source point (from differentiating Eq. 1)
        const cxf ywf = to_f(yw);
        const float sf = (float)L.s, m1f = (float)L.m1, m2f = (float)L.m2;
        float aR[5];
        cxf R[5];
#pragma unroll
        for (int i = 0; i < 5; i++) {
            const cxf d1 = inv(cxf{zf[i].x + sf, zf[i].y}), d2 = inv(zf[i]);
            R[i] = ywf - zf[i] + conj(m1f * d1 + m2f * d2);
            aR[i] = norm2(R[i]);
            cf1[i] = m1f * (d1 * d1) + m2f * (d2 * d2);
            const float J = 1.0f - norm2(cf1[i]);
            crJ[i] = 1.0f / (fabsf(J) < 1e-30f ? 1e-30f : J);
        }
        int r4 = 0, r5 = 0;
        float a3 = 0.f, a4 = 0.f, a5 = 0.f;
#pragma unroll
        for (int i = 0; i < 5; i++) {
            int r = 0;
#pragma unroll
            for (int j = 0; j < 5; j++)
                if (j != i) r += (aR[j] < aR[i]) || (aR[j] == aR[i] && j < i);
            if (r == 2) a3 = aR[i];
            if (r == 3) { r4 = i; a4 = aR[i]; }
            if (r == 4) { r5 = i; a5 = aR[i]; }
        }
        cxf R45 = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 5; i++)
            if (i == r4 || i == r5) R45 = R45 + R[i];
        if (norm2(R45) < 1e-4f * a5 && a4 > 100.0f * a3) cmask &= ~((1u << r4) | (1u << r5));
    }
    const float wx = (float)(yw.x - L.y0.x), wy = (float)(yw.y - L.y0.y), rhof = (float)L.rho;
#pragma unroll
    for (int t = 0; t < SPL; t++) {
        const int k = gl * SPL + t;
        const double th = twopi * k / SPI;
        cxd z[5] = {zc[0], zc[1], zc[2], zc[3], zc[4]};
        float sn, cs;
        sincosf((float)th, &sn, &cs);
        const cxf dzeta = {rhof * cs - wx, rhof * sn - wy};
        cxf dz[5];
#pragma unroll
        for (int i = 0; i < 5; i++) dz[i] = crJ[i] * (dzeta - conj(cf1[i]) * conj(dzeta));
        predict_roots(z, dz, cmask);
        flags |= limb_sample<PREC, RP>(L, th, z, ar, k, wc);
        ar.ordA[k] = (uint16_t)k;
    }
    co.sync();
#pragma unroll
    for (int t = 0; t < SPL; t++) {
        const int k = gl * SPL + t;
        const int ef = compute_edge(ar, k, (k + 1 == SPI) ? 0 : k + 1, twopi / SPI, &ar.eA[k], &ar.eE[k], true);
        if (ef & PS_SLOPE) vpos = k;
        xe = xe || (ef & EDGE_XING);
        wc.edges++;
    }
    co.sync();

    int N = SPI, nslot = SPI;
    uint16_t *ordA = ar.ordA, *ordB = ar.ordB;
    double A = 0.0, E = 0.0;
    for (;;) {
        // crossings of the last edges that failed the slope test (rare)
        if (REPAIR && W == 1) {
            if (__any_sync(FULL, vpos >= 0)) flags |= slope_repairs(ar, ordA, N, vpos);
        } else if (REPAIR) {
            // a repair re-judges samples and recomputes edges that the other
            // warps' lanes own: the warps of the group take turns, each turn
            // closed by a group barrier that every warp passes
            for (int w = 0; w < W; w++) {
                if (co.wig == w && __any_sync(FULL, vpos >= 0)) flags |= slope_repairs(ar, ordA, N, vpos);
                co.sync();
            }
        } else if (vpos >= 0) {
            flags |= PS_SLOPE;
        }
        vpos = -1;
        double a = 0.0, e = 0.0;
        for (int p = gl; p < N; p += 32 * W) {
            const int sl = ordA[p];
            a += ar.eA[sl];
            e += ar.eE[sl];
        }
        A = warp_sum(a);
        E = warp_sum(e);
        bool xing = __any_sync(FULL, xe);
        if (W > 1) {
            if (lane == 0) { co.ex[co.wig].a = A; co.ex[co.wig].e = E; co.ex[co.wig].xing = xing; }
            co.sync();
            A = 0.0;
            E = 0.0;
            xing = false;
#pragma unroll
            for (int w = 0; w < W; w++) { A += co.ex[w].a; E += co.ex[w].e; xing = xing || co.ex[w].xing; }
        }
        // Sec. 2.5: stop once the summed edge errors are within the tolerance
        // (a stricter target on limbs that cross a caustic, see XING_TOL_FACTOR)
        if (!(E > (xing ? XING_TOL_FACTOR : 1.0) * tol * fabs(A))) break;  // converged (or non-finite)
        if (nslot + SPI > cap) { flags |= PS_CAP; break; }

        // cumulative error in theta order, each edge less its share of the tolerance
        const double thr = tol * fabs(A) * rcp((double)N);
        const int chunk = (N + 32 * W - 1) / (32 * W);
        const int p0 = min(gl * chunk, N), p1 = min(p0 + chunk, N);
        double run = 0.0;
        for (int p = p0; p < p1; p++) {
            run += fmax(ar.eE[ordA[p]] - thr, 0.0);
            ar.cum[p] = run;
        }
        double incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        double Wsum = __shfl_sync(FULL, incl, 31);
        double excl = incl - run;
        if (W > 1) {
            // warp totals in group order: offsets of the later warps
            if (lane == 31) co.ex[co.wig].scan = incl;
            co.sync();
            double off = 0.0, tot = 0.0;
#pragma unroll
            for (int w = 0; w < W; w++) {
                const double v = co.ex[w].scan;
                if (w < co.wig) off += v;
                tot += v;
            }
            excl += off;
            Wsum = tot;
        }
        for (int p = p0; p < p1; p++) ar.cum[p] += excl;
        co.sync();

        // inverse transform at quantiles (j + 1/2)/SPI with linear interpolation
        double tn[SPL];
        int tp[SPL];
        bool tk[SPL];
#pragma unroll
        for (int t = 0; t < SPL; t++) {
            const int j = gl * SPL + t;
            const double target = (j + 0.5) * (Wsum / SPI);
            int lo = 0, hi = N - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (ar.cum[mid] > target) hi = mid; else lo = mid + 1;
            }
            const int sa = ordA[lo];
            const double wp = fmax(ar.eE[sa] - thr, 0.0);
            double frac = (wp > 0.0) ? (target - (ar.cum[lo] - wp)) * rcp(wp) : 0.5;
            frac = fmin(fmax(frac, 0.0), 1.0);
            const double ta = ar.theta[sa];
            const double tb = (lo + 1 < N) ? ar.theta[ordA[lo + 1]] : twopi;
            tn[t] = ta + frac * (tb - ta);
            tp[t] = lo;
            tk[t] = (tn[t] - ta > minsep) && (tb - tn[t] > minsep);
        }
        // drop a quantile that coincides with the previous one (the previous
        // warp's last quantile for the first lane of a warp of a group)
        double pth_w = 0.0;
        int ppos_w = -1;
        if (W > 1) {
            if (lane == 31) { co.ex[co.wig].last_th = tn[SPL - 1]; co.ex[co.wig].last_pos = tp[SPL - 1]; }
            co.sync();
            if (co.wig > 0) { pth_w = co.ex[co.wig - 1].last_th; ppos_w = co.ex[co.wig - 1].last_pos; }
        }
#pragma unroll
        for (int t = 0; t < SPL; t++) {
            double pth = __shfl_up_sync(FULL, tn[SPL - 1], 1);
            int ppos = __shfl_up_sync(FULL, tp[SPL - 1], 1);
            if (t > 0) { pth = tn[t - 1]; ppos = tp[t - 1]; }
            else if (W > 1 && lane == 0) { pth = pth_w; ppos = ppos_w; }
            const bool has_prev = (t > 0) || (gl > 0);
            if (has_prev && ppos == tp[t] && fabs(tn[t] - pth) <= minsep) tk[t] = false;
        }
        // compaction of the kept angles, in quantile order
        const unsigned lt = (1u << lane) - 1u;
        int before = 0, m = 0;
#pragma unroll
        for (int t = 0; t < SPL; t++) {
            const unsigned b = __ballot_sync(FULL, tk[t]);
            before += __popc(b & lt);
            m += __popc(b);
        }
        if (W > 1) {
            if (lane == 0) co.ex[co.wig].cnt = m;
            co.sync();
            int off = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < W; w++) {
                const int c = co.ex[w].cnt;
                if (w < co.wig) off += c;
                tot += c;
            }
            before += off;
            m = tot;
        }
        int rk[SPL];
        {
            int own = 0;
#pragma unroll
            for (int t = 0; t < SPL; t++) {
                rk[t] = before + own;
                own += tk[t] ? 1 : 0;
            }
        }
        if (m == 0) { flags |= PS_CAP; break; } // no room left between samples
#pragma unroll
        for (int t = 0; t < SPL; t++)
            if (tk[t]) {
                ws.theta_new[rk[t]] = tn[t];
                ws.pos_new[rk[t]] = (uint16_t)tp[t];
            }
        co.sync();

        // new samples, warm-started from the sample at the start of their interval
#pragma unroll
        for (int t = 0; t < SPL; t++)
            if (tk[t]) {
                const int sa = ordA[tp[t]];
                cxd z[5];
                cxf dz[5];
                const float dth = (float)(tn[t] - ar.theta[sa]);
#pragma unroll
                for (int i = 0; i < 5; i++) {
                    z[i] = ar.roots[sa * 5 + i];
                    dz[i] = dth * ar.zp[sa * 5 + i];
                }
                predict_roots(z, dz, real_mask(ar.meta[sa]));
                flags |= limb_sample<PREC, RP>(L, tn[t], z, ar, nslot + rk[t], wc);
            }
        // merge into theta order
        for (int p = p0; p < p1; p++) {
            int lo = 0, hi = m;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (ws.pos_new[mid] < p) lo = mid + 1; else hi = mid;
            }
            ordB[p + lo] = ordA[p];
        }
#pragma unroll
        for (int t = 0; t < SPL; t++)
            if (tk[t]) ordB[tp[t] + 1 + rk[t]] = (uint16_t)(nslot + rk[t]);
        co.sync();
        uint16_t *tmp = ordA; ordA = ordB; ordB = tmp;
        const int nslot_old = nslot;
        N += m;
        nslot += m;

        // edges touching the new samples
#pragma unroll
        for (int t = 0; t < SPL; t++)
            if (tk[t]) {
                const int P = tp[t] + 1 + rk[t];
                const int sl = nslot_old + rk[t];
                const int nx = (P + 1 < N) ? P + 1 : 0;
                const int sb = ordA[nx];
                const double tb = (P + 1 < N) ? ar.theta[sb] : twopi;
                int ef = compute_edge(ar, sl, sb, tb - tn[t], &ar.eA[sl], &ar.eE[sl], !xing);
                if (ef & PS_SLOPE) vpos = P;
                xe = xe || (ef & EDGE_XING);
                wc.edges++;
                const bool first = (rk[t] == 0) || (ws.pos_new[rk[t] - 1] != tp[t]);
                if (first) {
                    const int so = ordA[P - 1];
                    ef = compute_edge(ar, so, sl, tn[t] - ar.theta[so], &ar.eA[so], &ar.eE[so], !xing);
                    if (ef & PS_SLOPE) vpos = P - 1;
                    xe = xe || (ef & EDGE_XING);
                    wc.edges++;
                }
            }
        co.sync();

    }
    flags = __reduce_or_sync(FULL, flags);
    if (W > 1) {
        if (lane == 0) co.ex[co.wig].flags = flags;
        co.sync();
        flags = 0;
#pragma unroll
        for (int w = 0; w < W; w++) flags |= co.ex[w].flags;
        co.sync();
    }
    PosResult r;
    r.work.sw64 = __reduce_add_sync(FULL, wc.sw64);
    r.work.sw32 = __reduce_add_sync(FULL, wc.sw32);
    r.work.edges = __reduce_add_sync(FULL, wc.edges);
    r.work.nw64 = __reduce_add_sync(FULL, wc.nw64);
    r.area = A;
    r.err = E;
    r.nsamp = N;
    r.status = flags;
    return r;
}

}  // namespace tw
