/*
 * twinkle_oracle.c -- plain, slow CPU oracle for finite-source binary-lens
 * magnification of a uniform disc source.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline of the benchmark load this library; the GPU library never links,
 * includes or calls it, and it shares no code with it.
 *
 * What is computed (paper Sec. 1 and Sec. 2.3).  For a uniform source the
 * magnification is the total area of all images divided by the source area
 * pi*rho^2.  By Green's theorem (Eq. 8) each image area is a contour integral
 * of 1/2 z ^ dz along the image boundary; image boundaries are traced by the
 * images of the source limb zeta(theta) = zeta0 + rho e^{i theta}, and an image
 * of parity p = sign J (Eq. 7) is traversed counter-clockwise when p > 0 and
 * clockwise when p < 0 as theta increases (Sec. 2.3, discussion of Fig. 2).
 * Hence
 *
 *     A = Int_0^{2pi} 1/2 sum_{real images j} p_j  z_j ^ (dz_j/dtheta) dtheta.
 *
 * Unlike the contour method this never links images between samples: the limb
 * is cut at its caustic crossings (where the number of real images changes
 * between 3 and 5, Sec. 2.3), each piece is integrated by a double-exponential
 * (tanh-sinh) rule, and the pieces are added.  Near a crossing the two merging
 * images behave like zc +- a sqrt(theta - thetac); measured from the origin
 * their integrand has an inverse-square-root singularity whose weight is
 * |zc|*|a|, which no floating-point endpoint can resolve for small rho.  The
 * oracle therefore integrates each half of each piece about the critical
 * point zc of its crossing end:
 *
 *     Int 1/2 sum p (z - w) ^ dz  +  1/2 w ^ [S(end) - S(start)],
 *     S(theta) = sum_{real j} p_j z_j(theta)
 *
 * (an exact identity for any w).  S is continuous across a crossing (the two
 * merging images meet at zc with opposite parity), so the boundary terms at a
 * crossing cancel between its two sides and only the midpoint terms remain;
 * the integrand about zc is bounded (it vanishes like sqrt(theta - thetac)).
 *
 * Pieces of the method, each following the paper:
 *   - lens equation, centre-of-mass frame: Eq. 1-2 (Sec. 2.1);
 *   - quintic: built by generic polynomial arithmetic from Eq. 1 and its
 *     complex conjugate (NOT from the refactored coefficients of Eq. 6, which
 *     the GPU path uses);
 *   - roots: Laguerre iteration with deflation, then each root polished by
 *     Laguerre on the undeflated polynomial;
 *   - ghost images: residual of Eq. 12; ghosts come as a pair with opposite
 *     residuals (Sec. 2.4.1, consequence of Eq. 13-15);
 *   - parity and image derivative: Eq. 7 and dz/dtheta from differentiating
 *     Eq. 1 (Eq. 10 prints f' where its complex conjugate is meant);
 *   - real images refined by Newton's method on the lens equation itself
 *     (Eq. 1; conditioning 1/|J|) after classification: a root of the
 *     generically expanded quintic inside a cluster of roots next to a cusp
 *     is only good to eps B/|p'|, and that noise, amplified by 1/|J|, kept
 *     the quadrature from converging there;
 *   - caustic crossings: intersections of the limb with the caustic, the image
 *     of the critical curve J = 0 (Eq. 7), cross-checked by scanning the image
 *     count along the limb;
 *   - close approaches of the caustic to the limb that do not cross it (a
 *     limb grazing a cusp) split the quadrature as well: the point-source
 *     magnification peaks there with a width of about distance/rho.
 *
 * Arithmetic is long double throughout (x87 80-bit on x86-64, IEEE binary128
 * on AArch64).  The generic expansion is exposed to the catastrophic
 * cancellation of Sec. 2.2 at small q, which the extended precision absorbs.
 *
 * Status codes returned per position (see oracle/__init__.py):
 *   0 ok, 1 crossing detectors disagree / inconsistent image counts,
 *   2 quadrature did not reach its tolerance, 3 root finder failure,
 *   4 invalid input.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Working type: IEEE binary128 on both build hosts.  On x86-64 `long double`
 * is only the 64-bit-mantissa x87 format, which cannot resolve the near-double
 * roots next to a low-mass lens (q ~ 1e-9) from a generically expanded
 * polynomial, so GCC's __float128 is used there; on AArch64 Linux `long
 * double` already is binary128. */
#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 real;
typedef __complex128 cplx;
#define c_abs cabsq
#define c_sqrt csqrtq
#define c_conj conjq
#define c_re crealq
#define c_im cimagq
#define r_abs fabsq
#define r_atan2 atan2q
#define r_sinh sinhq
#define r_cosh coshq
#define r_exp expq
#define r_cos cosq
#define r_sin sinq
#define R_EPS FLT128_EPSILON
#define R_MAX FLT128_MAX
#define R_MANT FLT128_MANT_DIG
#define PI_L 3.141592653589793238462643383279502884Q
#else
#if LDBL_MANT_DIG != 113
#error "the oracle needs a binary128 long double on this host"
#endif
typedef long double real;
typedef long double _Complex cplx;
#define c_abs cabsl
#define c_sqrt csqrtl
#define c_conj conjl
#define c_re creall
#define c_im cimagl
#define r_abs fabsl
#define r_atan2 atan2l
#define r_sinh sinhl
#define r_cosh coshl
#define r_exp expl
#define r_cos cosl
#define r_sin sinl
#define R_EPS LDBL_EPSILON
#define R_MAX LDBL_MAX
#define R_MANT LDBL_MANT_DIG
#define PI_L 3.141592653589793238462643383279502884L
#endif

#define TWO_PI_L (2 * PI_L)

static inline cplx cmk(real re, real im) {
    cplx z;
    __real__ z = re;
    __imag__ z = im;
    return z;
}
static inline cplx c_expi(real t) { return cmk(r_cos(t), r_sin(t)); } /* e^{i t} */
static inline int r_finite(real x) { return r_abs(x) <= R_MAX; }

enum { ORC_OK = 0, ORC_XING = 1, ORC_QUAD = 2, ORC_ROOT = 3, ORC_INPUT = 4 };

static real eps_real(void) { return R_EPS; } /* unit round-off of the working type */

/* ------------------------------------------------------------------ lens */
/* Eq. 1-2: masses normalised to the total, q = m2/m1, origin at the centre
 * of mass, primary at -q s/(1+q), secondary at s/(1+q). */
typedef struct {
    real m1, m2;
    cplx z1, z2;
} lens_t;

static lens_t lens_make(real s, real q) {
    lens_t L;
    L.m1 = 1.0 / (1.0 + q);
    L.m2 = q / (1.0 + q);
    L.z1 = -q * s / (1.0 + q);
    L.z2 = s / (1.0 + q);
    return L;
}

/* f(z) of Eq. 7 and its first two derivatives. */
static void lens_f(const lens_t *L, cplx z, cplx *f, cplx *f1, cplx *f2) {
    cplx d1 = 1.0 / (L->z1 - z), d2 = 1.0 / (L->z2 - z);
    if (f) *f = L->m1 * d1 + L->m2 * d2;
    if (f1) *f1 = L->m1 * d1 * d1 + L->m2 * d2 * d2;
    if (f2) *f2 = 2.0 * (L->m1 * d1 * d1 * d1 + L->m2 * d2 * d2 * d2);
}

/* Eq. 1: source position of an image position. */
static cplx lens_map(const lens_t *L, cplx z) {
    cplx f;
    lens_f(L, z, &f, NULL, NULL);
    return z + c_conj(f);
}

/* ------------------------------------------------- polynomial arithmetic */
/* Coefficients are stored in ascending order: a[0] + a[1] z + ... */
static void poly_mul(const cplx *a, int da, const cplx *b, int db, cplx *c) {
    for (int i = 0; i <= da + db; i++) c[i] = 0;
    for (int i = 0; i <= da; i++)
        for (int j = 0; j <= db; j++) c[i + j] += a[i] * b[j];
}

/* Quintic whose roots contain the images of zeta.  From Eq. 1,
 *   conj(z) = conj(zeta) - m1/(z1 - z) - m2/(z2 - z) = N(z)/D(z),
 *   D = (z1 - z)(z2 - z);
 * substituting back into Eq. 1 gives zeta - z = m1 D/P1 + m2 D/P2 with
 * Pk = conj(zk) D - N, i.e.  (zeta - z) P1 P2 - m1 D P2 - m2 D P1 = 0. */
static void lens_quintic(const lens_t *L, cplx zeta, cplx c[6]) {
    const cplx a1[2] = {L->z1, -1.0}; /* z1 - z */
    const cplx a2[2] = {L->z2, -1.0}; /* z2 - z */
    cplx D[3], N[3], P1[3], P2[3], P12[5], DP1[5], DP2[5], t[6];
    poly_mul(a1, 1, a2, 1, D);
    for (int i = 0; i < 3; i++) N[i] = c_conj(zeta) * D[i];
    for (int i = 0; i < 2; i++) N[i] -= L->m1 * a2[i] + L->m2 * a1[i];
    for (int i = 0; i < 3; i++) {
        P1[i] = c_conj(L->z1) * D[i] - N[i];
        P2[i] = c_conj(L->z2) * D[i] - N[i];
    }
    poly_mul(P1, 2, P2, 2, P12);
    const cplx lin[2] = {zeta, -1.0};
    poly_mul(lin, 1, P12, 4, t);
    poly_mul(D, 2, P2, 2, DP2);
    poly_mul(D, 2, P1, 2, DP1);
    for (int i = 0; i < 6; i++) c[i] = t[i];
    for (int i = 0; i < 5; i++) c[i] -= L->m1 * DP2[i] + L->m2 * DP1[i];
}

/* Quartic whose roots are the critical-curve points with f'(z) = e^{i phi}:
 *   m1 (z2 - z)^2 + m2 (z1 - z)^2 - e^{i phi} (z1 - z)^2 (z2 - z)^2 = 0. */
static void crit_quartic(const lens_t *L, real phi, cplx c[5]) {
    const cplx a1[2] = {L->z1, -1.0};
    const cplx a2[2] = {L->z2, -1.0};
    cplx s1[3], s2[3], s12[5];
    poly_mul(a1, 1, a1, 1, s1);
    poly_mul(a2, 1, a2, 1, s2);
    poly_mul(s1, 2, s2, 2, s12);
    cplx e = c_expi(phi);
    for (int i = 0; i < 5; i++) c[i] = -e * s12[i];
    for (int i = 0; i < 3; i++) c[i] += L->m1 * s2[i] + L->m2 * s1[i];
}

/* Horner evaluation of p, p' and p''/2 at x. */
static void poly_eval(const cplx *a, int n, cplx x, cplx *p, cplx *dp, cplx *hd2p, real *bound) {
    cplx P = a[n], D1 = 0, D2 = 0;
    real ax = c_abs(x), b = c_abs(P);
    for (int j = n - 1; j >= 0; j--) {
        D2 = x * D2 + D1;
        D1 = x * D1 + P;
        P = x * P + a[j];
        b = c_abs(P) + ax * b;
    }
    *p = P;
    if (dp) *dp = D1;
    if (hd2p) *hd2p = D2;
    if (bound) *bound = b;
}

/* Laguerre's method for one root of the degree-n polynomial a, starting from
 * *x.  Returns the iteration count, or -1 when it did not converge.  Every
 * 16th step is shortened by a fixed irrational-ish factor so that the
 * iteration cannot settle into a cycle. */
static int laguerre(const cplx *a, int n, cplx *x) {
    const int maxit = 400;
    const real eps = eps_real();
    for (int it = 1; it <= maxit; it++) {
        cplx p, dp, hd2p;
        real bound;
        poly_eval(a, n, *x, &p, &dp, &hd2p, &bound);
        if (c_abs(p) <= 4.0 * eps * bound) return it; /* at round-off level */
        cplx G = dp / p;
        cplx H = G * G - 2.0 * hd2p / p;
        cplx sq = c_sqrt((real)(n - 1) * ((real)n * H - G * G));
        cplx gp = G + sq, gm = G - sq;
        if (c_abs(gm) > c_abs(gp)) gp = gm;
        cplx dx;
        if (c_abs(gp) > 0) dx = (real)n / gp;
        else dx = (1.0 + c_abs(*x)) * c_expi((real)it);
        cplx x1 = *x - dx;
        if (x1 == *x) return it;
        if (it % 16 == 0) *x = *x - 0.618 * dx;
        else *x = x1;
        if (c_abs(dx) <= 2.0 * eps * c_abs(*x)) return it;
    }
    return -1;
}

/* All n roots (n <= 5) of the polynomial a: Laguerre with deflation, then each
 * root re-converged by Laguerre on the undeflated polynomial.  If polishing
 * makes two roots coincide (a near-double root), the deflated values are kept
 * for that pair.  Returns 0 on success. */
static int poly_roots(const cplx *a, int n, cplx *roots) {
    cplx ad[6];
    for (int i = 0; i <= n; i++) ad[i] = a[i];
    for (int j = n; j >= 1; j--) {
        cplx x = 0;
        if (laguerre(ad, j, &x) < 0) {
            x = cmk(0.5, 0.3);
            if (laguerre(ad, j, &x) < 0) return -1;
        }
        roots[j - 1] = x;
        cplx rem = ad[j];
        for (int i = j - 1; i >= 0; i--) {
            cplx t = ad[i];
            ad[i] = rem;
            rem = t + x * rem;
        }
    }
    cplx pol[5];
    for (int j = 0; j < n; j++) {
        pol[j] = roots[j];
        if (laguerre(a, n, &pol[j]) < 0) pol[j] = roots[j];
    }
    for (int j = 0; j < n; j++) {
        int clash = 0;
        for (int k = 0; k < n; k++) {
            if (k == j) continue;
            real sep = c_abs(roots[j] - roots[k]);
            real sep_new = c_abs(pol[j] - pol[k]);
            if (sep_new < 1e-3 * sep) clash = 1;
        }
        if (!clash) roots[j] = pol[j];
    }
    for (int j = 0; j < n; j++)
        if (!r_finite(c_re(roots[j])) || !r_finite(c_im(roots[j]))) return -1;
    return 0;
}

/* ---------------------------------------------------- images of a point */
typedef struct {
    cplx r[5];     /* roots of the quintic */
    cplx R[5];     /* lens-equation residuals, Eq. 12 */
    int order[5];  /* root indices sorted by |R| ascending */
    int nreal_pair; /* 3 if the two largest residuals form a ghost pair, else 5 */
} point_t;

static int point_solve(const lens_t *L, cplx zeta, point_t *P) {
    cplx c[6];
    lens_quintic(L, zeta, c);
    if (poly_roots(c, 5, P->r) != 0) return ORC_ROOT;
    real a[5], noise[5];
    for (int i = 0; i < 5; i++) {
        cplx rb = c_conj(P->r[i]);
        P->R[i] = zeta - P->r[i] + L->m1 / (rb - c_conj(L->z1)) + L->m2 / (rb - c_conj(L->z2));
        a[i] = c_abs(P->R[i]);
        P->order[i] = i;
        /* Round-off level of this residual: a computed root is off by about
         * eps * B / |p'| (B the Horner bound of p at the root), and
         * R = zeta - r + conj f(r) moves by at most (1 + |f'|) times that. */
        cplx pv, dp, f1;
        real B;
        poly_eval(c, 5, P->r[i], &pv, &dp, NULL, &B);
        lens_f(L, P->r[i], NULL, &f1, NULL);
        noise[i] = R_EPS * B * (1 + c_abs(f1)) / c_abs(dp);
    }
    for (int i = 1; i < 5; i++) /* insertion sort by |R| */
        for (int k = i; k > 0 && a[P->order[k]] < a[P->order[k - 1]]; k--) {
            int t = P->order[k];
            P->order[k] = P->order[k - 1];
            P->order[k - 1] = t;
        }
    /* Sec. 2.4.1: ghosts, if any, are a pair whose residuals are equal and
     * opposite (they sum to minus the real residuals, ~ 0) and far above the
     * round-off level of those two roots.  The round-off gate matters next to
     * a critical curve, where a real pair is a near-double root whose residual
     * round-off is many times that of the other images. */
    int i4 = P->order[3], i5 = P->order[4];
    cplx R4 = P->R[i4], R5 = P->R[i5];
    real r3 = a[P->order[2]], r4 = a[i4], r5 = a[i5];
    real nz = noise[i4] > noise[i5] ? noise[i4] : noise[i5];
    int ghost = (c_abs(R4 + R5) < 1e-2 * r5) && (r4 > 1e3 * nz) && (r4 > 10 * r3);
    P->nreal_pair = ghost ? 3 : 5;
    return ORC_OK;
}

/* Jacobian (Eq. 7) at z. */
static real lens_jac(const lens_t *L, cplx z) {
    cplx f1;
    lens_f(L, z, NULL, &f1, NULL);
    return 1.0 - c_re(f1) * c_re(f1) - c_im(f1) * c_im(f1);
}

/* ------------------------------------------------------------- integrand */
typedef struct {
    lens_t L;
    cplx zeta0;
    real rho;
    int status;
    long nevals;
    long budget; /* integrand evaluations allowed before giving up refinement */
} ctx_t;

/* Newton refinement of a real image z of the source point zeta on the lens
 * equation itself (Eq. 1), after classification.  A root of the generically
 * expanded quintic inside a cluster of roots (several images and ghosts
 * within a small distance, next to a cusp) is only accurate to about
 * eps B/|p'(z)|, far above the round-off of Eq. 1, whose conditioning at an
 * image is 1/|J| (Eq. 7).  With R = zeta - z - conj(f(z)) (Eq. 12) the
 * linearised equation dz + conj(f') conj(dz) = R gives
 *     dz = (R - conj(f') conj(R)) / J.
 * A step is kept only while it lowers |R| and stays well inside the distance
 * `sep` to the nearest other root, so that no image is moved onto another. */
static cplx polish_image(const lens_t *L, cplx zeta, cplx z, real sep) {
    for (int it = 0; it < 4; it++) {
        cplx f, f1;
        lens_f(L, z, &f, &f1, NULL);
        cplx R = zeta - z - c_conj(f);
        real J = 1.0 - c_re(f1) * c_re(f1) - c_im(f1) * c_im(f1);
        if (J == 0 || c_abs(R) == 0) break;
        cplx dz = (R - c_conj(f1) * c_conj(R)) / J;
        if (!(c_abs(dz) < 0.1 * sep)) break;
        cplx zn = z + dz, fn;
        lens_f(L, zn, &fn, NULL, NULL);
        if (!(c_abs(zeta - zn - c_conj(fn)) < c_abs(R))) break;
        z = zn;
    }
    return z;
}

/* 1/2 sum_{real j} p_j (z_j - w) ^ dz_j/dtheta at limb angle theta, the real
 * images being the `count` roots of smallest residual, each refined on the
 * lens equation (polish_image).  With
 * dz/dtheta = (zeta' - conj(f') conj(zeta'))/J and p = sign J,
 * p (z - w) ^ z' = Im(conj(z - w) (zeta' - conj(f') conj(zeta'))) / |J|.
 * Optionally returns S = sum_j p_j z_j. */
static real integrand(ctx_t *X, real theta, int count, cplx w, cplx *S_out) {
    cplx e = c_expi(theta);
    cplx zeta = X->zeta0 + X->rho * e;
    cplx dzeta = cmk(0, 1) * X->rho * e;
    point_t P;
    X->nevals++;
    if (point_solve(&X->L, zeta, &P) != ORC_OK) {
        X->status = ORC_ROOT;
        return 0;
    }
    real g = 0;
    cplx S = 0;
    for (int k = 0; k < count; k++) {
        const int i = P.order[k];
        real sep = INFINITY;
        for (int j = 0; j < 5; j++)
            if (j != i && c_abs(P.r[j] - P.r[i]) < sep) sep = c_abs(P.r[j] - P.r[i]);
        cplx z = polish_image(&X->L, zeta, P.r[i], sep);
        cplx f1;
        lens_f(&X->L, z, NULL, &f1, NULL);
        real J = 1.0 - c_re(f1) * c_re(f1) - c_im(f1) * c_im(f1);
        if (J == 0) continue;
        cplx num = dzeta - c_conj(f1) * c_conj(dzeta);
        g += c_im(c_conj(z - w) * num) / r_abs(J);
        S += (J > 0 ? 1.0 : -1.0) * z;
    }
    if (S_out) *S_out = S;
    return 0.5 * g;
}

/* ----------------------------------------------------------- quadrature */
/* Tanh-sinh rule on [a, b]: x = c + h tanh(pi/2 sinh t).  Levels halve the
 * step; stop when two levels agree to tol (absolute).  Nodes are placed by
 * their distance to the nearer end so that nodes next to an end are exact.
 * Falls back to bisection of the interval when the level limit is reached. */
static real ts_rule(ctx_t *X, real a, real b, int count, cplx w, real tol, int depth) {
    const real tmax = 4.5;
    const int maxlev = 7;
    real c = 0.5 * (a + b), hw = 0.5 * (b - a);
    if (hw <= 0) return 0;
    real I_prev = 0, I_cur = 0;
    real h = 1.0;
    /* level 0 */
    {
        real sum = 0;
        for (int k = -(int)tmax; k <= (int)tmax; k++) {
            real t = (real)k * h;
            real u = 0.5 * PI_L * r_sinh(t);
            real ch = r_cosh(u);
            real wgt = hw * 0.5 * PI_L * r_cosh(t) / (ch * ch);
            real dist = hw * 2.0 / (r_exp(2.0 * r_abs(u)) + 1.0);
            real x = (t >= 0) ? b - dist : a + dist;
            if (dist <= 0) continue;
            sum += wgt * integrand(X, x, count, w, NULL);
        }
        I_cur = h * sum;
    }
    for (int lev = 1; lev <= maxlev; lev++) {
        h *= 0.5;
        real sum = 0;
        int kmax = (int)(tmax / h);
        for (int k = -kmax; k <= kmax; k++) {
            if (!(k & 1)) continue; /* only the nodes new at this level */
            real t = (real)k * h;
            real u = 0.5 * PI_L * r_sinh(t);
            real ch = r_cosh(u);
            real wgt = hw * 0.5 * PI_L * r_cosh(t) / (ch * ch);
            real dist = hw * 2.0 / (r_exp(2.0 * r_abs(u)) + 1.0);
            real x = (t >= 0) ? b - dist : a + dist;
            if (dist <= 0) continue;
            sum += wgt * integrand(X, x, count, w, NULL);
        }
        I_prev = I_cur;
        I_cur = 0.5 * I_prev + h * sum;
        if (lev >= 3 && r_abs(I_cur - I_prev) <= tol) return I_cur;
    }
    if (depth <= 0 || X->nevals > X->budget) {
        X->status = X->status ? X->status : ORC_QUAD;
        return I_cur;
    }
    return ts_rule(X, a, c, count, w, 0.5 * tol, depth - 1) +
           ts_rule(X, c, b, count, w, 0.5 * tol, depth - 1);
}

/* Periodic trapezoid rule over the full limb (no crossings): spectrally
 * convergent for a smooth periodic integrand; doubles the node count until two
 * levels agree.  Falls back to tanh-sinh on eight arcs. */
static real periodic_rule(ctx_t *X, int count, real tol) {
    int n = 64;
    real sum = 0;
    for (int k = 0; k < n; k++) sum += integrand(X, TWO_PI_L * k / n, count, 0, NULL);
    real I_cur = TWO_PI_L * sum / n;
    while (n < 16384) {
        real add = 0;
        for (int k = 0; k < n; k++) add += integrand(X, TWO_PI_L * (2 * k + 1) / (2 * n), count, 0, NULL);
        sum += add;
        n *= 2;
        real I_new = TWO_PI_L * sum / n;
        if (r_abs(I_new - I_cur) <= tol && n >= 256) return I_new;
        I_cur = I_new;
    }
    real tot = 0;
    for (int k = 0; k < 8; k++)
        tot += ts_rule(X, TWO_PI_L * k / 8, TWO_PI_L * (k + 1) / 8, count, 0, tol / 8, 10);
    return tot;
}

/* ------------------------------------------------- critical curve/caustic */
typedef struct {
    int M;
    cplx *zc; /* M x 4 critical points, columns tracked by continuity in phi */
    cplx *cc; /* their caustic images */
    int wrap[4]; /* column at phi = 0 continuing column b at phi = 2 pi */
    int ok;
} crit_t;

static const int PERM4[24][4] = {
    {0,1,2,3},{0,1,3,2},{0,2,1,3},{0,2,3,1},{0,3,1,2},{0,3,2,1},
    {1,0,2,3},{1,0,3,2},{1,2,0,3},{1,2,3,0},{1,3,0,2},{1,3,2,0},
    {2,0,1,3},{2,0,3,1},{2,1,0,3},{2,1,3,0},{2,3,0,1},{2,3,1,0},
    {3,0,1,2},{3,0,2,1},{3,1,0,2},{3,1,2,0},{3,2,0,1},{3,2,1,0}};

static int best_perm4(const cplx *prev, const cplx *cur) {
    int best = 0;
    real bd = INFINITY;
    for (int p = 0; p < 24; p++) {
        real d = 0;
        for (int b = 0; b < 4; b++) d += c_abs(cur[PERM4[p][b]] - prev[b]);
        if (d < bd) { bd = d; best = p; }
    }
    return best;
}

static int crit_build(const lens_t *L, int M, crit_t *C) {
    C->M = M;
    C->zc = (cplx *)malloc(sizeof(cplx) * 4 * M);
    C->cc = (cplx *)malloc(sizeof(cplx) * 4 * M);
    C->ok = 1;
    if (!C->zc || !C->cc) { C->ok = 0; return -1; }
    cplx q[5], r[4];
    for (int k = 0; k < M; k++) {
        crit_quartic(L, TWO_PI_L * k / M, q);
        if (poly_roots(q, 4, r) != 0) { C->ok = 0; return -1; }
        if (k == 0) {
            for (int b = 0; b < 4; b++) C->zc[b] = r[b];
        } else {
            int p = best_perm4(&C->zc[4 * (k - 1)], r);
            for (int b = 0; b < 4; b++) C->zc[4 * k + b] = r[PERM4[p][b]];
        }
        for (int b = 0; b < 4; b++) C->cc[4 * k + b] = lens_map(L, C->zc[4 * k + b]);
    }
    int p = best_perm4(&C->zc[4 * (M - 1)], &C->zc[0]);
    for (int b = 0; b < 4; b++) C->wrap[b] = PERM4[p][b];
    return 0;
}

static void crit_free(crit_t *C) {
    free(C->zc);
    free(C->cc);
}

/* Critical point at angle phi on the branch passing near `guess`. */
static cplx crit_point(const lens_t *L, real phi, cplx guess) {
    cplx q[5], r[4];
    crit_quartic(L, phi, q);
    if (poly_roots(q, 4, r) != 0) return guess;
    int bi = 0;
    for (int b = 1; b < 4; b++)
        if (c_abs(r[b] - guess) < c_abs(r[bi] - guess)) bi = b;
    return r[bi];
}

typedef struct {
    real theta;  /* limb angle of the crossing, in [0, 2pi) */
    cplx zc;     /* critical point whose caustic image is on the limb */
} xing_t;

#define MAX_XING 64

static real limb_dist(const lens_t *L, cplx zeta0, real rho, cplx z) {
    return c_abs(lens_map(L, z) - zeta0) - rho;
}

static void add_xing(xing_t *xs, int *nx, const lens_t *L, cplx zeta0, cplx zc) {
    if (*nx >= MAX_XING) return;
    cplx d = lens_map(L, zc) - zeta0;
    real th = r_atan2(c_im(d), c_re(d));
    if (th < 0) th += TWO_PI_L;
    xs[*nx].theta = th;
    xs[*nx].zc = zc;
    (*nx)++;
}

/* Bisection of a sign change of the limb distance between (pa, za) and
 * (pb, zb) on one tracked branch. */
static cplx bisect_branch(const lens_t *L, cplx zeta0, real rho, real pa, cplx za, real pb, cplx zb) {
    real da = limb_dist(L, zeta0, rho, za);
    for (int it = 0; it < 90; it++) {
        real pm = 0.5 * (pa + pb);
        if (pm == pa || pm == pb) break;
        cplx zm = crit_point(L, pm, 0.5 * (za + zb));
        real dm = limb_dist(L, zeta0, rho, zm);
        if ((dm < 0) == (da < 0)) { pa = pm; za = zm; da = dm; }
        else { pb = pm; zb = zm; }
    }
    return 0.5 * (za + zb);
}

/* Limb angle of the point nearest to zc (the direction of zc from the source
 * centre). */
static real limb_angle(cplx zeta0, cplx zc) {
    cplx d = zc - zeta0;
    real th = r_atan2(c_im(d), c_re(d));
    return th < 0 ? th + TWO_PI_L : th;
}

/* A close approach of the caustic to the limb, closer than NEAR_FRAC * rho,
 * makes the point-source magnification along the limb peak sharply (width
 * about distance/rho in angle) where no image count changes; its angle is
 * recorded as a split point of the quadrature (tanh-sinh resolves features at
 * the end of an interval, not inside it). */
#define NEAR_FRAC 0.05
#define MAX_SPLIT 64

/* Method (ii): limb/caustic intersections.  Sign changes of the limb distance
 * along each tracked branch are bisected; local minima of |distance| that do
 * not change sign between grid points are searched (golden section) for a
 * pair of crossings hidden inside one grid cell.  Minima that stay on one side
 * but come within NEAR_FRAC * rho of the limb are returned in splits[] (limb
 * angles, *nsplit of them) when splits is not NULL. */
static int crossings_caustic(const lens_t *L, const crit_t *C, cplx zeta0, real rho, xing_t *xs, real *splits,
                             int *nsplit) {
    int nx = 0, M = C->M;
    if (nsplit) *nsplit = 0;
    real *d = (real *)malloc(sizeof(real) * 4 * M);
    if (!d) return -1;
    for (int i = 0; i < 4 * M; i++) d[i] = c_abs(C->cc[i] - zeta0) - rho;
    for (int b = 0; b < 4; b++) {
        for (int k = 0; k < M; k++) {
            int kn = (k + 1) % M;
            int bn = (k + 1 < M) ? b : C->wrap[b];
            real pa = TWO_PI_L * k / M, pb = TWO_PI_L * (k + 1) / M;
            cplx za = C->zc[4 * k + b], zb = C->zc[4 * kn + bn];
            real da = d[4 * k + b], db = d[4 * kn + bn];
            if ((da < 0) != (db < 0)) {
                add_xing(xs, &nx, L, zeta0, bisect_branch(L, zeta0, rho, pa, za, pb, zb));
                continue;
            }
            /* local minimum of |d| at k on this branch? */
            int kp = (k + M - 1) % M;
            int bp = b;
            if (k == 0) { /* predecessor column at phi = 2pi - step */
                for (int c = 0; c < 4; c++) if (C->wrap[c] == b) bp = c;
            }
            real dp = d[4 * kp + bp];
            if (!((dp < 0) == (da < 0) && r_abs(da) <= r_abs(dp) && r_abs(da) <= r_abs(db))) continue;
            const int near = splits && r_abs(da) < 4.0 * NEAR_FRAC * rho;
            /* skip minima whose parabola through the three grid values stays
             * well away from zero (unless the approach is close) */
            real curv = dp - 2.0 * da + db;
            if (curv != 0 && !near) {
                real vmin = da - (db - dp) * (db - dp) / (8.0 * curv);
                if (r_abs(vmin) > 0.5 * r_abs(da) && (vmin < 0) == (da < 0)) continue;
            }
            /* golden-section search of sgn*d on [phi_{k-1}, phi_{k+1}] */
            real sg = (da < 0) ? -1.0 : 1.0;
            real lo = TWO_PI_L * (k - 1) / M, hi = TWO_PI_L * (k + 1) / M;
            cplx zlo = C->zc[4 * kp + bp], zhi = zb, zmid = za;
            const real gr = 0.6180339887498948482;
            real x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
            cplx g1 = crit_point(L, x1, zmid), g2 = crit_point(L, x2, zmid);
            real f1 = sg * limb_dist(L, zeta0, rho, g1), f2 = sg * limb_dist(L, zeta0, rho, g2);
            int found = 0;
            real pmin = 0;
            cplx zmin = 0;
            for (int it = 0; it < 80; it++) {
                if (f1 < 0 || f2 < 0) {
                    found = 1;
                    if (f1 < 0) { pmin = x1; zmin = g1; } else { pmin = x2; zmin = g2; }
                    break;
                }
                if (f1 < f2) { hi = x2; x2 = x1; g2 = g1; f2 = f1; x1 = hi - gr * (hi - lo); g1 = crit_point(L, x1, g2); f1 = sg * limb_dist(L, zeta0, rho, g1); }
                else { lo = x1; x1 = x2; g1 = g2; f1 = f2; x2 = lo + gr * (hi - lo); g2 = crit_point(L, x2, g1); f2 = sg * limb_dist(L, zeta0, rho, g2); }
                if (hi - lo < 1e-17) break;
            }
            if (found) {
                real plo = TWO_PI_L * (k - 1) / M, phi_hi = TWO_PI_L * (k + 1) / M;
                add_xing(xs, &nx, L, zeta0, bisect_branch(L, zeta0, rho, plo, zlo, pmin, zmin));
                add_xing(xs, &nx, L, zeta0, bisect_branch(L, zeta0, rho, pmin, zmin, phi_hi, zhi));
            } else if (near) {
                /* no crossing: the closest approach is a split point */
                real fm = f1 < f2 ? f1 : f2;
                cplx zm = f1 < f2 ? g1 : g2;
                if (fm < NEAR_FRAC * rho && *nsplit < MAX_SPLIT) splits[(*nsplit)++] = limb_angle(zeta0, lens_map(L, zm));
            }
        }
    }
    free(d);
    /* sort by angle and merge duplicates */
    for (int i = 1; i < nx; i++)
        for (int k = i; k > 0 && xs[k].theta < xs[k - 1].theta; k--) {
            xing_t t = xs[k]; xs[k] = xs[k - 1]; xs[k - 1] = t;
        }
    int m = 0;
    for (int i = 0; i < nx; i++) {
        if (m > 0 && r_abs(xs[i].theta - xs[m - 1].theta) < 1e-13) continue;
        xs[m++] = xs[i];
    }
    if (m >= 2 && TWO_PI_L - xs[m - 1].theta + xs[0].theta < 1e-13) m--;
    return m;
}

/* Image count along the limb by the residual pair test. */
static int count_at(ctx_t *X, real theta) {
    point_t P;
    cplx zeta = X->zeta0 + X->rho * c_expi(theta);
    X->nevals++;
    if (point_solve(&X->L, zeta, &P) != ORC_OK) { X->status = ORC_ROOT; return 5; }
    return P.nreal_pair;
}

/* Method (i): changes of the image count on a uniform grid of K limb angles,
 * each bisected to full precision.  A change is kept only if the count
 * differs between the two sides at 1e-10 and 1e-8 rad from it: where many
 * images sit next to a critical curve, the residual test can misjudge an
 * isolated angle, and bisection can settle on such a point instead of the
 * crossing.  Returns the number found. */
static int crossings_scan(ctx_t *X, int K, real *out, int maxout) {
    int n = 0;
    int c0 = count_at(X, 0), cprev = c0;
    for (int k = 1; k <= K; k++) {
        real th = TWO_PI_L * k / K;
        int c = (k == K) ? c0 : count_at(X, th);
        if (c != cprev) {
            real a = TWO_PI_L * (k - 1) / K, b = th;
            for (int it = 0; it < 70; it++) {
                real m = 0.5 * (a + b);
                if (m == a || m == b) break;
                if (count_at(X, m) == cprev) a = m; else b = m;
            }
            real x = 0.5 * (a + b);
            int real_change = 1;
            for (real dd = 1e-10; dd < 2e-8; dd *= 100)
                if (count_at(X, x - dd) == count_at(X, x + dd)) real_change = 0;
            if (real_change) {
                if (n < maxout) out[n] = x;
                n++;
            }
        }
        cprev = c;
    }
    return n;
}

/* -------------------------------------------------------- magnification */
typedef struct {
    int status;
    int nxing;
    long nevals;
} mag_info_t;

/* Integral over one piece [a, b] of the limb (b > a) with `count` images,
 * whose ends are crossings with critical points wa (at a) and wb (at b).
 * Interior split angles sp[0..ns-1] (ascending, inside (a, b)) cut it into
 * sub-arcs: the first is integrated about wa, the last about wb, the others
 * about the origin; with none, the piece is cut at its midpoint.  For a
 * sub-arc [u, v] integrated about w,
 *   Int 1/2 sum p z ^ dz = Int 1/2 sum p (z - w) ^ dz + 1/2 w ^ [S(v) - S(u)],
 * and the terms at the crossings cancel against the neighbouring pieces (S is
 * continuous there and both sides use the same w), so what is added here is
 * 1/2 wa ^ S(first cut) - 1/2 wb ^ S(last cut). */
static real piece_integral(ctx_t *X, real a, real b, int count, cplx wa, cplx wb, const real *sp, int ns, real tol) {
    real mid = 0.5 * (a + b);
    real c0 = ns ? sp[0] : mid, c1 = ns ? sp[ns - 1] : mid;
    real tsub = tol / (ns + 2);
    real A = ts_rule(X, a, c0, count, wa, tsub, 40);
    for (int k = 0; k + 1 < ns; k++) A += ts_rule(X, sp[k], sp[k + 1], count, 0, tsub, 40);
    A += ts_rule(X, c1, b, count, wb, tsub, 40);
    cplx S0, S1;
    (void)integrand(X, c0, count, 0, &S0);
    (void)integrand(X, c1, count, 0, &S1);
    A += 0.5 * (c_re(wa) * c_im(S0) - c_im(wa) * c_re(S0));
    A -= 0.5 * (c_re(wb) * c_im(S1) - c_im(wb) * c_re(S1));
    return A;
}

/* Area of a limb cut at nx >= 2 crossings xs (ascending angles, each with its
 * critical point), each piece between consecutive crossings integrated by
 * piece_integral with the split angles sp[0..nsp-1] that fall inside it.
 * Sets X->status to ORC_XING unless consecutive pieces alternate between 3
 * and 5 images. */
static real pieces_area(ctx_t *X, const xing_t *xs, int nx, const real *sp, int nsp, real tol) {
    real A = 0;
    int counts[MAX_XING];
    for (int i = 0; i < nx; i++) {
        real a = xs[i].theta;
        real b = (i + 1 < nx) ? xs[i + 1].theta : xs[0].theta + TWO_PI_L;
        real mid = 0.5 * (a + b);
        counts[i] = count_at(X, mid);
        cplx wa = xs[i].zc, wb = xs[(i + 1) % nx].zc;
        /* split angles strictly inside the piece */
        real ins[MAX_SPLIT];
        int nin = 0;
        for (int k = 0; k < nsp; k++) {
            real t = sp[k] < a ? sp[k] + TWO_PI_L : sp[k];
            if (t > a + 1e-12 * (b - a) && t < b - 1e-12 * (b - a)) ins[nin++] = t;
        }
        for (int u = 1; u < nin; u++)
            for (int k = u; k > 0 && ins[k] < ins[k - 1]; k--) {
                real t = ins[k]; ins[k] = ins[k - 1]; ins[k - 1] = t;
            }
        A += piece_integral(X, a, b, counts[i], wa, wb, ins, nin, tol);
    }
    /* consecutive pieces must alternate between 3 and 5 images */
    for (int i = 0; i < nx; i++) {
        int c = counts[i], cn = counts[(i + 1) % nx];
        if (!((c == 3 && cn == 5) || (c == 5 && cn == 3))) X->status = ORC_XING;
    }
    return A;
}

/* Critical point of a crossing at limb angle th found by the image-count
 * scan: at a fold the two images that merge there sit at zc +- a sqrt(d) +
 * b d a small angle d inside the five-image side, so their midpoint is zc to
 * O(d).  Returns 0 when neither side of th shows five images. */
static int scan_crit_point(ctx_t *X, real th, cplx *zc) {
    const real d = 1e-16;
    for (int side = -1; side <= 1; side += 2) {
        point_t P;
        cplx zeta = X->zeta0 + X->rho * c_expi(th + side * d);
        X->nevals++;
        if (point_solve(&X->L, zeta, &P) != ORC_OK || P.nreal_pair != 5) continue;
        int bi = 0, bj = 1;
        real best = c_abs(P.r[0] - P.r[1]);
        for (int i = 0; i < 5; i++)
            for (int j = i + 1; j < 5; j++)
                if (c_abs(P.r[i] - P.r[j]) < best) { best = c_abs(P.r[i] - P.r[j]); bi = i; bj = j; }
        *zc = 0.5 * (P.r[bi] + P.r[bj]);
        return 1;
    }
    return 0;
}

static real mag_one(const lens_t *L, const crit_t *C, real y1, real y2, real rho, int scan_K, mag_info_t *info) {
    ctx_t X;
    X.L = *L;
    X.zeta0 = cmk(y1, y2);
    X.rho = rho;
    X.status = ORC_OK;
    X.nevals = 0;
    X.budget = 1000000;
    xing_t xs[MAX_XING];
    real sp[MAX_SPLIT];
    int nsp = 0;
    int nx = crossings_caustic(L, C, X.zeta0, rho, xs, sp, &nsp);
    if (nx < 0) nx = 0;
    if (nx % 2) X.status = ORC_XING;
    for (int i = 1; i < nsp; i++) /* split angles in ascending order */
        for (int k = i; k > 0 && sp[k] < sp[k - 1]; k--) {
            real t = sp[k]; sp[k] = sp[k - 1]; sp[k - 1] = t;
        }
    /* absolute tolerance: 1e-12 of the source area, per piece */
    real tol = 1e-12 * PI_L * rho * rho;
    real A = 0;
    if (nx < 2 && nsp == 0) {
        int count = count_at(&X, 0);
        A = periodic_rule(&X, count, tol);
    } else if (nx < 2) {
        /* no crossing, close approaches: tanh-sinh over the arcs between them */
        int count = count_at(&X, sp[0]);
        for (int k = 0; k < nsp; k++) {
            real a = sp[k], b = (k + 1 < nsp) ? sp[k + 1] : sp[0] + TWO_PI_L;
            if (b - a > 1e-30) A += ts_rule(&X, a, b, count, 0, tol / nsp, 40);
        }
    } else {
        A = pieces_area(&X, xs, nx, sp, nsp, tol);
    }
    if (scan_K > 0 && X.status == ORC_OK) {
        real sc[MAX_XING];
        int ns = crossings_scan(&X, scan_K, sc, MAX_XING);
        /* every crossing seen by the scan must be one the caustic search found */
        if (ns > MAX_XING) X.status = ORC_XING;
        for (int i = 0; i < ns && i < MAX_XING; i++) {
            int match = 0;
            for (int k = 0; k < nx; k++) {
                real dd = r_abs(sc[i] - xs[k].theta);
                if (dd > PI_L) dd = TWO_PI_L - dd;
                if (dd < 1e-8) match = 1;
            }
            if (!match) X.status = ORC_XING;
        }
    }
    /* Crossings the caustic search missed (a cusp tip reaching into the limb
     * between its caustic samples) leave the quadrature unconverged or the
     * detectors in disagreement.  The crossings are then the image-count
     * changes themselves (Sec. 2.3), found by a scan of 4096 limb angles,
     * each bisected, with critical points from the merging image pairs; the
     * limb is integrated again on them and the result kept if it converges
     * with alternating image counts. */
    if (X.status == ORC_QUAD || X.status == ORC_XING) {
        ctx_t Y = X;
        Y.status = ORC_OK;
        Y.nevals = 0;
        real sc[MAX_XING];
        int ns = crossings_scan(&Y, 4096, sc, MAX_XING);
        if (Y.status == ORC_OK && ns >= 2 && ns % 2 == 0 && ns <= MAX_XING) {
            xing_t ys[MAX_XING];
            int ok = 1;
            for (int i = 0; i < ns && ok; i++) {
                ys[i].theta = sc[i];
                ok = scan_crit_point(&Y, sc[i], &ys[i].zc);
            }
            if (ok) {
                real A2 = pieces_area(&Y, ys, ns, sp, nsp, tol);
                if (Y.status == ORC_OK) {
                    A = A2;
                    X.status = ORC_OK;
                    nx = ns;
                }
            }
        }
        X.nevals += Y.nevals;
    }
    if (info) {
        info->status = X.status;
        info->nxing = nx;
        info->nevals = X.nevals;
    }
    return A / (PI_L * rho * rho);
}

/* ====================================================== exported API ===== */

/* Coefficients (ascending, interleaved re/im) of the quintic of one source
 * position, in the centre-of-mass frame. */
void orc_quintic(double s, double q, double zr, double zi, double *out12) {
    lens_t L = lens_make(s, q);
    cplx c[6];
    lens_quintic(&L, cmk(zr, zi), c);
    for (int i = 0; i < 6; i++) {
        out12[2 * i] = (double)c_re(c[i]);
        out12[2 * i + 1] = (double)c_im(c[i]);
    }
}

/* Images of one point source: roots (re/im), residuals (re/im), Jacobians, a
 * real-image mask, and the image count from the residual pair test.  Returns
 * 0 or a status code. */
int orc_images(double s, double q, double zr, double zi, double *roots10, double *res10, double *jac5,
               int32_t *isreal5, int32_t *count) {
    lens_t L = lens_make(s, q);
    point_t P;
    int st = point_solve(&L, cmk(zr, zi), &P);
    if (st) return st;
    for (int i = 0; i < 5; i++) {
        roots10[2 * i] = (double)c_re(P.r[i]);
        roots10[2 * i + 1] = (double)c_im(P.r[i]);
        res10[2 * i] = (double)c_re(P.R[i]);
        res10[2 * i + 1] = (double)c_im(P.R[i]);
        jac5[i] = (double)lens_jac(&L, P.r[i]);
        isreal5[i] = 0;
    }
    for (int k = 0; k < P.nreal_pair; k++) isreal5[P.order[k]] = 1;
    *count = P.nreal_pair;
    return 0;
}

/* Critical curve and caustic sampled at M angles (4 branches each). */
int orc_caustic(double s, double q, int M, double *zc8M, double *cc8M) {
    lens_t L = lens_make(s, q);
    crit_t C;
    if (crit_build(&L, M, &C) != 0) { crit_free(&C); return ORC_ROOT; }
    for (int i = 0; i < 4 * M; i++) {
        zc8M[2 * i] = (double)c_re(C.zc[i]);
        zc8M[2 * i + 1] = (double)c_im(C.zc[i]);
        cc8M[2 * i] = (double)c_re(C.cc[i]);
        cc8M[2 * i + 1] = (double)c_im(C.cc[i]);
    }
    crit_free(&C);
    return 0;
}

/* Crossing angles of one limb by method 1 (caustic, returns n) or method 2
 * (image-count scan on K points). */
int orc_crossings(double s, double q, double rho, double y1, double y2, int method, int K, double *out, int maxout) {
    lens_t L = lens_make(s, q);
    if (method == 1) {
        crit_t C;
        if (crit_build(&L, K, &C) != 0) { crit_free(&C); return -1; }
        xing_t xs[MAX_XING];
        int n = crossings_caustic(&L, &C, cmk(y1, y2), rho, xs, NULL, NULL);
        for (int i = 0; i < n && i < maxout; i++) out[i] = (double)xs[i].theta;
        crit_free(&C);
        return n;
    }
    ctx_t X;
    X.L = L;
    X.zeta0 = cmk(y1, y2);
    X.rho = rho;
    X.status = 0;
    X.nevals = 0;
    X.budget = 400000;
    real tmp[MAX_XING];
    int n = crossings_scan(&X, K, tmp, MAX_XING);
    for (int i = 0; i < n && i < maxout && i < MAX_XING; i++) out[i] = (double)tmp[i];
    return n;
}

/* Close approaches of the caustic to one limb that do not cross it (limb
 * angles, at most maxout); returns their number.  These are the split points
 * of the quadrature in mag_one. */
int orc_close_approaches(double s, double q, double rho, double y1, double y2, double *out, int maxout) {
    lens_t L = lens_make(s, q);
    crit_t C;
    if (crit_build(&L, 4096, &C) != 0) { crit_free(&C); return -1; }
    xing_t xs[MAX_XING];
    real sp[MAX_SPLIT];
    int nsp = 0;
    (void)crossings_caustic(&L, &C, cmk(y1, y2), rho, xs, sp, &nsp);
    for (int i = 0; i < nsp && i < maxout; i++) out[i] = (double)sp[i];
    crit_free(&C);
    return nsp;
}

/* Finite-source magnifications of n positions sharing one lens and source
 * radius.  status[i] receives the position's status code, nxing[i] the
 * number of caustic crossings of its limb (either may be NULL).  scan_K > 0
 * cross-checks the crossings by an image-count scan on scan_K limb points.
 * nthreads <= 0 uses the OpenMP default.  Returns 0, or ORC_INPUT. */
int orc_mag(double s, double q, double rho, const double *y1, const double *y2, int64_t n, int scan_K,
            int nthreads, double *out, int32_t *status, int32_t *nxing) {
    if (!(s > 0) || !(q > 0) || !(rho > 0) || n < 0) return ORC_INPUT;
    lens_t L = lens_make(s, q);
    crit_t C;
    if (crit_build(&L, 4096, &C) != 0) {
        crit_free(&C);
        for (int64_t i = 0; i < n; i++) { out[i] = NAN; if (status) status[i] = ORC_ROOT; }
        return 0;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < n; i++) {
        mag_info_t info;
        out[i] = (double)mag_one(&L, &C, y1[i], y2[i], rho, scan_K, &info);
        if (status) status[i] = info.status;
        if (nxing) nxing[i] = info.nxing;
    }
    crit_free(&C);
    return 0;
}

/* Radii (below rmax, ascending, at most maxout; returns their number) at
 * which the circle |zeta - zeta0| = r changes the way it meets the caustic,
 * where the uniform-disc magnification mu(r) is not smooth: the local
 * extrema of the distance from zeta0 along each caustic branch (the circle
 * touches a fold there; refined by golden-section search on the branch
 * parameter) and the distances of the cusps (where the caustic point stalls:
 * a local minimum of its speed along the branch below a thousandth of the
 * branch's median speed). */
int orc_singular_radii(double s, double q, double y1, double y2, double rmax, double *out, int maxout) {
    lens_t L = lens_make(s, q);
    crit_t C;
    const int M = 4096;
    if (crit_build(&L, M, &C) != 0) { crit_free(&C); return -1; }
    cplx z0 = cmk(y1, y2);
    int n = 0;
    real *d = (real *)malloc(sizeof(real) * M), *v = (real *)malloc(sizeof(real) * M), *vs = (real *)malloc(sizeof(real) * M);
    if (!d || !v || !vs) { free(d); free(v); free(vs); crit_free(&C); return -1; }
    for (int b = 0; b < 4; b++) {
        /* the branch in order, continued through the wrap as crossings_caustic does */
        cplx *zb = (cplx *)malloc(sizeof(cplx) * M);
        for (int k = 0; k < M; k++) zb[k] = C.zc[4 * k + b];
        for (int k = 0; k < M; k++) d[k] = c_abs(lens_map(&L, zb[k]) - z0);
        for (int k = 0; k + 1 < M; k++) v[k] = c_abs(lens_map(&L, zb[k + 1]) - lens_map(&L, zb[k]));
        v[M - 1] = v[M - 2];
        for (int k = 0; k < M; k++) vs[k] = v[k];
        for (int i = 1; i < M; i++) /* median speed: insertion sort of a copy */
            for (int k = i; k > 0 && vs[k] < vs[k - 1]; k--) { real t = vs[k]; vs[k] = vs[k - 1]; vs[k - 1] = t; }
        const real vmed = vs[M / 2];
        for (int k = 1; k + 1 < M; k++) {
            const real pa = TWO_PI_L * (k - 1) / M, pb = TWO_PI_L * (k + 1) / M;
            if ((d[k] - d[k - 1]) * (d[k + 1] - d[k]) < 0 && n < maxout) {
                /* extremum of the distance: golden-section search */
                const real sg = d[k] < d[k - 1] ? 1.0 : -1.0; /* minimise sg * d */
                real lo = pa, hi = pb;
                const real gr = 0.6180339887498948482;
                real x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
                cplx g1 = crit_point(&L, x1, zb[k]), g2 = crit_point(&L, x2, zb[k]);
                real f1 = sg * c_abs(lens_map(&L, g1) - z0), f2 = sg * c_abs(lens_map(&L, g2) - z0);
                for (int it = 0; it < 90 && hi - lo > 1e-30; it++) {
                    if (f1 < f2) { hi = x2; x2 = x1; f2 = f1; x1 = hi - gr * (hi - lo); g1 = crit_point(&L, x1, zb[k]); f1 = sg * c_abs(lens_map(&L, g1) - z0); }
                    else { lo = x1; x1 = x2; f1 = f2; x2 = lo + gr * (hi - lo); g2 = crit_point(&L, x2, zb[k]); f2 = sg * c_abs(lens_map(&L, g2) - z0); }
                }
                const real r = sg * (f1 < f2 ? f1 : f2);
                if (r < rmax) out[n++] = (double)r;
            }
            if (v[k] < v[k - 1] && v[k] <= v[k + 1] && v[k] < 1e-3 * vmed && n < maxout) {
                const real r = c_abs(lens_map(&L, zb[k]) - z0); /* a cusp */
                if (r < rmax) out[n++] = (double)r;
            }
        }
        free(zb);
    }
    free(d); free(v); free(vs);
    crit_free(&C);
    for (int i = 1; i < n; i++)
        for (int k = i; k > 0 && out[k] < out[k - 1]; k--) { double t = out[k]; out[k] = out[k - 1]; out[k - 1] = t; }
    return n;
}

/* Uniform-disc magnifications of one source position for n radii (the caustic
 * is built once): the annuli of a limb-darkened source.  status[i] as in
 * orc_mag.  Returns 0, or ORC_INPUT. */
int orc_mag_radii(double s, double q, double y1, double y2, const double *radii, int64_t n, int scan_K, int nthreads,
                  double *out, int32_t *status) {
    if (!(s > 0) || !(q > 0) || n < 0) return ORC_INPUT;
    lens_t L = lens_make(s, q);
    crit_t C;
    if (crit_build(&L, 4096, &C) != 0) {
        crit_free(&C);
        for (int64_t i = 0; i < n; i++) { out[i] = NAN; if (status) status[i] = ORC_ROOT; }
        return 0;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < n; i++) {
        mag_info_t info;
        out[i] = radii[i] > 0 ? (double)mag_one(&L, &C, y1, y2, radii[i], scan_K, &info) : NAN;
        if (status) status[i] = radii[i] > 0 ? info.status : ORC_INPUT;
    }
    crit_free(&C);
    return 0;
}

/* Source trajectory of a light curve (a straight line; the paper leaves the
 * convention open): tau = (t - t0)/tE,
 *   y1 = tau cos(alpha) - u0 sin(alpha),  y2 = tau sin(alpha) + u0 cos(alpha). */
void orc_trajectory(double u0, double alpha, double t0, double tE, const double *t, int64_t n, double *y1,
                    double *y2) {
    for (int64_t i = 0; i < n; i++) {
        real tau = ((real)t[i] - t0) / tE;
        y1[i] = (double)(tau * r_cos(alpha) - u0 * r_sin(alpha));
        y2[i] = (double)(tau * r_sin(alpha) + u0 * r_cos(alpha));
    }
}

/* Brute-force inverse ray shooting (Sec. 1): rays from the centres of an
 * nx x ny grid of image-plane pixels over [x0,x1] x [y0,y1] are mapped by
 * Eq. 1; the magnification is (pixel area x rays landing in the disc) / its
 * area.  Independent of everything above except the lens equation itself. */
double orc_rayshoot(double s, double q, double rho, double y1, double y2, double x0, double x1, double yb0,
                    double yb1, int64_t nx, int64_t ny, int nthreads) {
    double m1 = 1.0 / (1.0 + q), m2 = q / (1.0 + q);
    double z1 = -q * s / (1.0 + q), z2 = s / (1.0 + q);
    double dx = (x1 - x0) / nx, dy = (yb1 - yb0) / ny;
    int64_t hits = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for reduction(+ : hits) schedule(static)
#endif
    for (int64_t j = 0; j < ny; j++) {
        double y = yb0 + (j + 0.5) * dy;
        int64_t h = 0;
        for (int64_t i = 0; i < nx; i++) {
            double x = x0 + (i + 0.5) * dx;
            /* zeta = z + m1/(conj z1 - conj z) + m2/(conj z2 - conj z), lenses on the real axis */
            double ax = z1 - x, bx = z2 - x;         /* conj(zk) - conj(z) = (zk - x) + i y */
            double d1 = ax * ax + y * y, d2 = bx * bx + y * y;
            double zr = x + m1 * ax / d1 + m2 * bx / d2;
            double zi = y - m1 * y / d1 - m2 * y / d2;
            double ex = zr - y1, ey = zi - y2;
            if (ex * ex + ey * ey < rho * rho) h++;
        }
        hits += h;
    }
    return (double)hits * dx * dy / (M_PI * rho * rho);
}

/* Sizes of the working type, for the Python side to report. */
int orc_real_bits(void) { return (int)R_MANT; }
