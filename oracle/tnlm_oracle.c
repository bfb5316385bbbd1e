/*
 * FP64 CPU oracle of the TNLM 4DCT reconstruction path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA library; the two meet only through the seeded inputs.
 *
 * It is plain and slow on purpose: every function follows one passage of
 * the paper (arXiv:1009.1351) in the paper's order and notation, with no
 * blocking, fusion or reordering beyond what that passage states.
 *
 *   orc_project / orc_backproject   P_i and P_i^T (Sec. 2.1, Eq. 1): the
 *       system matrix entry A[r][j] is the length of ray r inside pixel j,
 *       traced by Siddon's parametric plane-crossing method (the ray tracer
 *       the paper names in Sec. 3).
 *   orc_cgls                        the CGLS box of Sec. 2.2, per phase.
 *   orc_grad_step                   Eq. 4 (plain gradient data step).
 *   orc_weights                     Eq. 8 with the normalisation of Eq. 3
 *       (sum over y of omega = 1), search window of Sec. 2.3.
 *   orc_gj                          the Gauss-Jacobi box of Sec. 2.2.
 *   orc_reconstruct                 the TNLM algorithm box of Sec. 2.2.
 *   orc_fbp                         step 1 of the TNLM box: FBP of all views
 *   orc_objective_op                data term of Eq. 1 plus the TNLM energy
 *       whose exact prox the Gauss-Jacobi fixed point (Eq. 7) is.
 *   orc_tnlm_term, orc_data_term    the two terms of Eq. 1 (J as Eq. 2).
 *
 * Readings where the paper is silent (kept identical on the CUDA side):
 *   - pixel squares are [c - d/2, c + d/2) on each axis; a segment is given
 *     to the pixel containing its midpoint;
 *   - patches take the value 0 outside the image (zero extension);
 *   - the window W x W includes the zero shift and only candidates y inside
 *     the image take part (in the sum and in Z);
 *   - Eq. 8 is evaluated as exp(-(D - min D)/h^2) / sum(...), equal to
 *     exp(-D/h^2)/Z in exact arithmetic;
 *   - Jacobi ordering: every phase uses the previous sweep's neighbours;
 *   - CGLS scalars a, b are per phase; the last step's s update is unused
 *     and skipped; a zero denominator stops that phase's CGLS;
 *   - the clamp f = max(f, 0) is applied after Gauss-Jacobi only.
 *
 * Layouts: images f[phase][iy][ix] (ix fastest), sinograms q[phase][view][bin].
 * Geometry: ints gi = {nx, ny, N, V, B}, doubles gd = {pixel, bin_mm, sid, sdd},
 * angles[N*V] = source angle of every view (radians).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NX   gi[0]
#define NY   gi[1]
#define NPH  gi[2]
#define NV   gi[3]
#define NB   gi[4]
#define PIX  gd[0]
#define BINW gd[1]
#define SID  gd[2]
#define SDD  gd[3]

static const double ORC_PI = 3.14159265358979323846;

int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Ray geometry: source S and detector point E of ray (phase, view, bin).    */
/* ------------------------------------------------------------------------ */
static void ray_of(const int* gi, const double* gd, const double* ang, long ray,
                   double* sx, double* sy, double* ex, double* ey)
{
    long b = ray % NB;
    long gv = ray / NB;                 /* phase * V + view */
    double th = ang[gv];
    double gam = ((double)b - 0.5 * (NB - 1)) * (BINW / SDD);
    double cx = -cos(th), cy = -sin(th);           /* central ray direction */
    double ux = cx * cos(gam) - cy * sin(gam);     /* rotate by gamma (ccw) */
    double uy = cx * sin(gam) + cy * cos(gam);
    *sx = SID * cos(th);
    *sy = SID * sin(th);
    *ex = *sx + SDD * ux;
    *ey = *sy + SDD * uy;
}

/* Siddon traversal: lists (pixel index, length in mm) of one ray.
 * Returns the count.  cap must be >= nx + ny + 2. */
static int siddon(const int* gi, const double* gd, double sx, double sy, double ex, double ey,
                  long* idx, double* len, double* work)
{
    const int nx = NX, ny = NY;
    const double dl = PIX;
    const double x0 = -0.5 * nx * dl, y0 = -0.5 * ny * dl;
    const double dx = ex - sx, dy = ey - sy;
    const double d12 = sqrt(dx * dx + dy * dy);
    double amin = 0.0, amax = 1.0;
    if (dx != 0.0) {
        double a0 = (x0 - sx) / dx, a1 = (x0 + nx * dl - sx) / dx;
        amin = fmax(amin, fmin(a0, a1));
        amax = fmin(amax, fmax(a0, a1));
    } else if (sx < x0 || sx >= x0 + nx * dl) {
        return 0;
    }
    if (dy != 0.0) {
        double a0 = (y0 - sy) / dy, a1 = (y0 + ny * dl - sy) / dy;
        amin = fmax(amin, fmin(a0, a1));
        amax = fmin(amax, fmax(a0, a1));
    } else if (sy < y0 || sy >= y0 + ny * dl) {
        return 0;
    }
    if (!(amax > amin)) return 0;

    /* crossings of the x- and y-planes strictly inside (amin, amax), each
     * list sorted ascending, then merged. */
    double* ax_ = work;
    double* ay_ = work + (nx + 1);
    double* al = work + (nx + 1) + (ny + 1);
    int nxa = 0, nya = 0;
    if (dx != 0.0) {
        for (int k = 0; k <= nx; ++k) {
            int kk = dx > 0 ? k : nx - k;
            double a = (x0 + kk * dl - sx) / dx;
            if (a > amin && a < amax) ax_[nxa++] = a;
        }
    }
    if (dy != 0.0) {
        for (int k = 0; k <= ny; ++k) {
            int kk = dy > 0 ? k : ny - k;
            double a = (y0 + kk * dl - sy) / dy;
            if (a > amin && a < amax) ay_[nya++] = a;
        }
    }
    int na = 0, p = 0, q = 0;
    al[na++] = amin;
    while (p < nxa || q < nya) {
        if (q >= nya || (p < nxa && ax_[p] <= ay_[q])) al[na++] = ax_[p++];
        else al[na++] = ay_[q++];
    }
    al[na++] = amax;

    int n = 0;
    for (int m = 1; m < na; ++m) {
        double a_lo = al[m - 1], a_hi = al[m];
        if (!(a_hi > a_lo)) continue;
        double am = 0.5 * (a_lo + a_hi);
        double px = sx + am * dx, py = sy + am * dy;
        long ix = (long)floor((px - x0) / dl);
        long iy = (long)floor((py - y0) / dl);
        if (ix < 0 || ix >= nx || iy < 0 || iy >= ny) continue;
        idx[n] = iy * nx + ix;
        len[n] = (a_hi - a_lo) * d12;
        ++n;
    }
    return n;
}

/* One ray's non-zero system-matrix entries (for dense checks in tests). */
int orc_ray_entries(const int* gi, const double* gd, const double* ang, long ray,
                    long* idx, double* len)
{
    double sx, sy, ex, ey;
    double* work = (double*)malloc(sizeof(double) * (3 * (NX + NY) + 8));
    ray_of(gi, gd, ang, ray, &sx, &sy, &ex, &ey);
    int n = siddon(gi, gd, sx, sy, ex, ey, idx, len, work);
    free(work);
    return n;
}

/* (P f)_{i,v,b} = sum_j A[(i,v,b)][j] f_i[j] */
void orc_project(const int* gi, const double* gd, const double* ang, const double* f, double* q)
{
    const long nrays = (long)NPH * NV * NB;
    const long npx = (long)NX * NY;
#pragma omp parallel
    {
        long* idx = (long*)malloc(sizeof(long) * (NX + NY + 4));
        double* len = (double*)malloc(sizeof(double) * (NX + NY + 4));
        double* work = (double*)malloc(sizeof(double) * (3 * (NX + NY) + 8));
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < nrays; ++r) {
            double sx, sy, ex, ey;
            ray_of(gi, gd, ang, r, &sx, &sy, &ex, &ey);
            int n = siddon(gi, gd, sx, sy, ex, ey, idx, len, work);
            const double* fi = f + (r / ((long)NV * NB)) * npx;
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += len[k] * fi[idx[k]];
            q[r] = acc;
        }
        free(idx); free(len); free(work);
    }
}

/* (P^T q)_i[j] = sum_{v,b} A[(i,v,b)][j] q_{i,v,b}: serial scatter per phase. */
void orc_backproject(const int* gi, const double* gd, const double* ang, const double* q, double* f)
{
    const long npx = (long)NX * NY;
    const long rays_per_phase = (long)NV * NB;
    memset(f, 0, sizeof(double) * npx * NPH);
#pragma omp parallel
    {
        long* idx = (long*)malloc(sizeof(long) * (NX + NY + 4));
        double* len = (double*)malloc(sizeof(double) * (NX + NY + 4));
        double* work = (double*)malloc(sizeof(double) * (3 * (NX + NY) + 8));
#pragma omp for schedule(static, 1)
        for (int i = 0; i < NPH; ++i) {
            double* fi = f + (long)i * npx;
            for (long rr = 0; rr < rays_per_phase; ++rr) {
                long r = (long)i * rays_per_phase + rr;
                double sx, sy, ex, ey;
                ray_of(gi, gd, ang, r, &sx, &sy, &ex, &ey);
                int n = siddon(gi, gd, sx, sy, ex, ey, idx, len, work);
                for (int k = 0; k < n; ++k) fi[idx[k]] += len[k] * q[r];
            }
        }
        free(idx); free(len); free(work);
    }
}

/* ------------------------------------------------------------------------ */
/* Data step.                                                                */
/* ------------------------------------------------------------------------ */
static double dot(const double* a, const double* b, long n)
{
    double s = 0.0;
    for (long k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* CGLS box (Sec. 2.2) for every phase i, with P_ni = Sigma^{-1/2} P_i and
 * y_ni = Sigma^{-1/2} y_i, Sigma^{-1} = w (diagonal).  u holds f^(k-1) on
 * entry and g^(k) = u^(M1) on exit.  res0 (may be NULL) receives, per
 * phase, ||r^(0)||^2 = ||Sigma^{-1/2}(y_i - P_i f_i^(k-1))||^2. */
void orc_cgls(const int* gi, const double* gd, const double* ang,
              const double* y, const double* w, double* u, int m1, double* res0)
{
    const long npx = (long)NX * NY, nsg = (long)NV * NB;
    const long NI = npx * NPH, NS = nsg * NPH;
    double* r = (double*)malloc(sizeof(double) * NS);
    double* t = (double*)malloc(sizeof(double) * NS);
    double* s = (double*)malloc(sizeof(double) * NI);
    double* gr = (double*)malloc(sizeof(double) * NI);
    double* gam = (double*)malloc(sizeof(double) * NPH);
    double* a = (double*)malloc(sizeof(double) * NPH);
    int* active = (int*)malloc(sizeof(int) * NPH);

    /* r0 = y_n - P_n u0 ; s0 = P_n^T r0 */
    orc_project(gi, gd, ang, u, t);
    for (long k = 0; k < NS; ++k) r[k] = sqrt(w[k]) * (y[k] - t[k]);
    for (long k = 0; k < NS; ++k) t[k] = sqrt(w[k]) * r[k];
    orc_backproject(gi, gd, ang, t, s);
    for (int i = 0; i < NPH; ++i) {
        if (res0) res0[i] = dot(r + i * nsg, r + i * nsg, nsg);
        gam[i] = dot(s + i * npx, s + i * npx, npx);      /* ||P_n^T r^(0)||^2 */
        active[i] = 1;
    }
    for (int m = 0; m < m1; ++m) {
        /* step 1: a = ||P_n^T r||^2 / ||P_n s||^2 */
        orc_project(gi, gd, ang, s, t);
        for (long k = 0; k < NS; ++k) t[k] *= sqrt(w[k]);          /* P_n s */
        for (int i = 0; i < NPH; ++i) {
            double den = dot(t + i * nsg, t + i * nsg, nsg);
            if (!active[i] || den == 0.0 || gam[i] == 0.0) { active[i] = 0; a[i] = 0.0; }
            else a[i] = gam[i] / den;
        }
        /* steps 2-3 */
        for (int i = 0; i < NPH; ++i) {
            if (!active[i]) continue;
            for (long k = 0; k < npx; ++k) u[i * npx + k] += a[i] * s[i * npx + k];
            for (long k = 0; k < nsg; ++k) r[i * nsg + k] -= a[i] * t[i * nsg + k];
        }
        if (m == m1 - 1) break;                 /* s^(M1) would be unused */
        /* steps 4-5: b = ||P_n^T r^(m+1)||^2 / ||P_n^T r^(m)||^2, s update */
        for (long k = 0; k < NS; ++k) t[k] = sqrt(w[k]) * r[k];
        orc_backproject(gi, gd, ang, t, gr);
        for (int i = 0; i < NPH; ++i) {
            if (!active[i]) continue;
            double gnew = dot(gr + i * npx, gr + i * npx, npx);
            double b = gnew / gam[i];
            for (long k = 0; k < npx; ++k) s[i * npx + k] = gr[i * npx + k] + b * s[i * npx + k];
            gam[i] = gnew;
        }
    }
    free(r); free(t); free(s); free(gr); free(gam); free(a); free(active);
}

/* Eq. 4: g = f - (1/beta) P^T Sigma^{-1} (P f - y). */
void orc_grad_step(const int* gi, const double* gd, const double* ang,
                   const double* y, const double* w, const double* f, double beta, double* g,
                   double* res0)
{
    const long npx = (long)NX * NY, nsg = (long)NV * NB;
    const long NI = npx * NPH, NS = nsg * NPH;
    double* t = (double*)malloc(sizeof(double) * NS);
    orc_project(gi, gd, ang, f, t);
    if (res0)
        for (int i = 0; i < NPH; ++i) {
            double s = 0.0;
            for (long k = i * nsg; k < (i + 1) * nsg; ++k) s += w[k] * (t[k] - y[k]) * (t[k] - y[k]);
            res0[i] = s;
        }
    for (long k = 0; k < NS; ++k) t[k] = w[k] * (t[k] - y[k]);
    orc_backproject(gi, gd, ang, t, g);
    for (long k = 0; k < NI; ++k) g[k] = f[k] - g[k] / beta;
    free(t);
}

/* ------------------------------------------------------------------------ */
/* TNLM weights, Eq. 8.                                                      */
/* ------------------------------------------------------------------------ */
static double pix0(const double* img, int nx, int ny, int x, int y)
{
    return (x < 0 || x >= nx || y < 0 || y >= ny) ? 0.0 : img[(long)y * nx + x];
}

/* ||R_{g_i}(x) - R_{g_j}(y)||_2^2 over a d x d patch, zero extension. */
static double patch_dist(const double* gi_, const double* gj_, int nx, int ny,
                         int x0, int y0, int x1, int y1, int r)
{
    double s = 0.0;
    for (int py = -r; py <= r; ++py)
        for (int px = -r; px <= r; ++px) {
            double e = pix0(gi_, nx, ny, x0 + px, y0 + py) - pix0(gj_, nx, ny, x1 + px, y1 + py);
            s += e * e;
        }
    return s;
}

/* Normalised weights of Eq. 8 for both neighbours of every phase.
 *   wnext[i][iy][ix][sig] = omega_{i,i+1}(x, x+sig)
 *   wprev[i][iy][ix][sig] = omega_{i,i-1}(x, x+sig)
 *   dnext[i][iy][ix][sig] = ||R_{g_i}(x) - R_{g_{i+1}}(x+sig)||^2 (or +inf when
 *                           x+sig is outside the image); may be NULL.
 * sig = (sy + rho) * W + (sx + rho), rho = (W-1)/2.  Phase indices are cyclic. */
void orc_weights(int N, int nx, int ny, const double* g, int d, int W, double h,
                 double* wnext, double* wprev, double* dnext)
{
    const int r = (d - 1) / 2, rho = (W - 1) / 2, W2 = W * W;
    const long npx = (long)nx * ny;
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < N; ++i)
        for (long p = 0; p < npx; ++p) {
            int x = (int)(p % nx), yy = (int)(p / nx);
            double* dl = (double*)malloc(sizeof(double) * W2);
            for (int dir = 0; dir < 2; ++dir) {
                int j = dir == 0 ? (i + 1) % N : (i + N - 1) % N;
                double* out = (dir == 0 ? wnext : wprev) + ((long)i * npx + p) * W2;
                const double* gii = g + (long)i * npx;
                const double* gjj = g + (long)j * npx;
                double dmin = INFINITY;
                for (int sy = -rho; sy <= rho; ++sy)
                    for (int sx = -rho; sx <= rho; ++sx) {
                        int k = (sy + rho) * W + (sx + rho);
                        int x1 = x + sx, y1 = yy + sy;
                        if (x1 < 0 || x1 >= nx || y1 < 0 || y1 >= ny) { dl[k] = INFINITY; continue; }
                        dl[k] = patch_dist(gii, gjj, nx, ny, x, yy, x1, y1, r);
                        if (dl[k] < dmin) dmin = dl[k];
                    }
                if (dir == 0 && dnext)
                    for (int k = 0; k < W2; ++k) dnext[((long)i * npx + p) * W2 + k] = dl[k];
                double z = 0.0;
                for (int k = 0; k < W2; ++k) {
                    double e = isinf(dl[k]) ? 0.0 : exp(-(dl[k] - dmin) / (h * h));
                    out[k] = e;
                    z += e;
                }
                for (int k = 0; k < W2; ++k) out[k] /= z;
            }
            free(dl);
        }
}

/* ------------------------------------------------------------------------ */
/* Gauss-Jacobi box (Sec. 2.2): u^(0) = g,                                   */
/* u_i^(m+1)(x) = g_i(x)/(mu+1) + mu/(2mu+2) [ sum_y u_{i-1}^(m)(y) w_{i,i-1}(x,y) */
/*                                           + sum_y u_{i+1}^(m)(y) w_{i,i+1}(x,y) ] */
/* ------------------------------------------------------------------------ */
void orc_gj(int N, int nx, int ny, int W, const double* g, const double* wnext,
            const double* wprev, double mu_hat, int m2, double* u_out)
{
    const int rho = (W - 1) / 2, W2 = W * W;
    const long npx = (long)nx * ny, NI = npx * N;
    double* u = (double*)malloc(sizeof(double) * NI);
    double* un = (double*)malloc(sizeof(double) * NI);
    memcpy(u, g, sizeof(double) * NI);
    for (int m = 0; m < m2; ++m) {
#pragma omp parallel for collapse(2) schedule(static)
        for (int i = 0; i < N; ++i)
            for (long p = 0; p < npx; ++p) {
                int x = (int)(p % nx), yy = (int)(p / nx);
                const double* up = u + (long)((i + N - 1) % N) * npx;
                const double* unx = u + (long)((i + 1) % N) * npx;
                const double* wp = wprev + ((long)i * npx + p) * W2;
                const double* wn = wnext + ((long)i * npx + p) * W2;
                double sp = 0.0, sn = 0.0;
                for (int sy = -rho; sy <= rho; ++sy)
                    for (int sx = -rho; sx <= rho; ++sx) {
                        int k = (sy + rho) * W + (sx + rho);
                        int x1 = x + sx, y1 = yy + sy;
                        if (x1 < 0 || x1 >= nx || y1 < 0 || y1 >= ny) continue;
                        sp += up[(long)y1 * nx + x1] * wp[k];
                        sn += unx[(long)y1 * nx + x1] * wn[k];
                    }
                un[(long)i * npx + p] = g[(long)i * npx + p] / (mu_hat + 1.0)
                                      + mu_hat / (2.0 * mu_hat + 2.0) * (sp + sn);
            }
        double* tmp = u; u = un; un = tmp;
    }
    memcpy(u_out, u, sizeof(double) * NI);
    free(u); free(un);
}

/* ------------------------------------------------------------------------ */
/* TNLM algorithm box (Sec. 2.2).                                            */
/*   ip = {d, W, m1, m2, K, data_step (0 CGLS, 1 Eq. 4), clamp}              */
/*   dp = {mu_hat, h, beta}                                                  */
/* f: in f^(0), out f^(K).  frozen_wnext/prev: if non-NULL, these weights    */
/* are used in every iteration instead of Eq. 8 (for fixed-point tests).     */
/* hist_rel[k] = ||f^(k) - f^(k-1)|| / ||f^(k)||, hist_res[k] = data term of */
/* f^(k-1) (sum over phases); either may be NULL.                            */
/* ------------------------------------------------------------------------ */
void orc_reconstruct(const int* gi, const double* gd, const double* ang,
                     const double* y, const double* w, double* f,
                     const int* ip, const double* dp,
                     const double* frozen_wnext, const double* frozen_wprev,
                     double* hist_rel, double* hist_res)
{
    const int d = ip[0], W = ip[1], m1 = ip[2], m2 = ip[3], K = ip[4], step = ip[5], clamp = ip[6];
    const double mu_hat = dp[0], h = dp[1], beta = dp[2];
    const long npx = (long)NX * NY, NI = npx * NPH;
    const long W2 = (long)W * W;
    double* g = (double*)malloc(sizeof(double) * NI);
    double* fn = (double*)malloc(sizeof(double) * NI);
    double* res = (double*)malloc(sizeof(double) * NPH);
    double* wn = frozen_wnext ? NULL : (double*)malloc(sizeof(double) * NI * W2);
    double* wp = frozen_wprev ? NULL : (double*)malloc(sizeof(double) * NI * W2);
    for (int k = 0; k < K; ++k) {
        /* step 2: data step from f^(k-1) */
        if (step == 0) {
            memcpy(g, f, sizeof(double) * NI);
            orc_cgls(gi, gd, ang, y, w, g, m1, res);
        } else {
            orc_grad_step(gi, gd, ang, y, w, f, beta, g, res);
        }
        /* step 3: weights from g^(k) */
        const double* use_n = frozen_wnext;
        const double* use_p = frozen_wprev;
        if (!frozen_wnext || !frozen_wprev) {
            orc_weights(NPH, NX, NY, g, d, W, h, wn, wp, NULL);
            use_n = wn; use_p = wp;
        }
        /* step 4: Gauss-Jacobi */
        orc_gj(NPH, NX, NY, W, g, use_n, use_p, mu_hat, m2, fn);
        /* step 5: positivity */
        if (clamp)
            for (long q = 0; q < NI; ++q) if (fn[q] < 0.0) fn[q] = 0.0;
        double dn = 0.0, nn = 0.0, rs = 0.0;
        for (long q = 0; q < NI; ++q) { dn += (fn[q] - f[q]) * (fn[q] - f[q]); nn += fn[q] * fn[q]; }
        for (int i = 0; i < NPH; ++i) rs += res[i];
        if (hist_rel) hist_rel[k] = nn > 0.0 ? sqrt(dn / nn) : 0.0;
        if (hist_res) hist_res[k] = rs;
        memcpy(f, fn, sizeof(double) * NI);
    }
    free(g); free(fn); free(res); free(wn); free(wp);
}

/* E_op(f) = sum_i (P_i f_i - y_i)^T w (P_i f_i - y_i)
 *         + mu * sum_i [ ||f_i||^2 - <f_i, W_{i,i+1} f_{i+1}> ]
 * with W_{i,i+1} given by wnext (the prox of mu * [...] with step 1/(2 beta)
 * has the Gauss-Jacobi fixed point of Eq. 7 when W_{i+1,i} = W_{i,i+1}^T). */
double orc_objective_op(const int* gi, const double* gd, const double* ang,
                        const double* y, const double* w, const double* f,
                        const double* wnext, int W, double mu)
{
    const long npx = (long)NX * NY, NS = (long)NPH * NV * NB;
    const int rho = (W - 1) / 2, W2 = W * W;
    double* t = (double*)malloc(sizeof(double) * NS);
    orc_project(gi, gd, ang, f, t);
    double data = 0.0;
    for (long k = 0; k < NS; ++k) data += w[k] * (t[k] - y[k]) * (t[k] - y[k]);
    double reg = 0.0;
    for (int i = 0; i < NPH; ++i) {
        const double* fi = f + (long)i * npx;
        const double* fj = f + (long)((i + 1) % NPH) * npx;
        for (long p = 0; p < npx; ++p) {
            int x = (int)(p % NX), yy = (int)(p / NX);
            double wf = 0.0;
            for (int sy = -rho; sy <= rho; ++sy)
                for (int sx = -rho; sx <= rho; ++sx) {
                    int x1 = x + sx, y1 = yy + sy;
                    if (x1 < 0 || x1 >= NX || y1 < 0 || y1 >= NY) continue;
                    wf += wnext[((long)i * npx + p) * W2 + (sy + rho) * W + (sx + rho)] * fj[(long)y1 * NX + x1];
                }
            reg += fi[p] * fi[p] - fi[p] * wf;
        }
    }
    free(t);
    return data + mu * reg;
}

/* The bracket of Eq. 1 summed over phases, each J as Eq. 2 defines it:
 *   T(f) = sum_i [ J(f_i, f_{i-1}) + J(f_i, f_{i+1}) ],
 *   J(f_i, f_j) = sum_x sum_y [f_i(x) - f_j(y)]^2 omega_{i,j}(x, y),
 * with omega_{i,i+1}(x, x+s) = wnext[i][x][s] and omega_{i,i-1}(x, x+s) =
 * wprev[i][x][s] (rows over the W x W window, candidates outside the image
 * carry no weight).  Eq. 1 is then data + (mu / 2) * T(f). */
double orc_tnlm_term(int N, int nx, int ny, int W, const double* f, const double* wnext,
                     const double* wprev)
{
    const int rho = (W - 1) / 2, W2 = W * W;
    const long npx = (long)nx * ny;
    double tot = 0.0;
    for (int i = 0; i < N; ++i) {
        const double* fi = f + (long)i * npx;
        for (int dir = 0; dir < 2; ++dir) {
            const int j = dir == 0 ? (i + N - 1) % N : (i + 1) % N;
            const double* fj = f + (long)j * npx;
            const double* w = dir == 0 ? wprev : wnext;
            double J = 0.0;
            for (long p = 0; p < npx; ++p) {
                int x = (int)(p % nx), yy = (int)(p / nx);
                for (int sy = -rho; sy <= rho; ++sy)
                    for (int sx = -rho; sx <= rho; ++sx) {
                        int x1 = x + sx, y1 = yy + sy;
                        if (x1 < 0 || x1 >= nx || y1 < 0 || y1 >= ny) continue;
                        double dv = fi[p] - fj[(long)y1 * nx + x1];
                        J += dv * dv * w[((long)i * npx + p) * W2 + (sy + rho) * W + (sx + rho)];
                    }
            }
            tot += J;
        }
    }
    return tot;
}

/* Data term of Eq. 1: sum_i (P_i f_i - y_i)^T Sigma^{-1} (P_i f_i - y_i). */
double orc_data_term(const int* gi, const double* gd, const double* ang, const double* y,
                     const double* w, const double* f)
{
    const long NS = (long)NPH * NV * NB;
    double* t = (double*)malloc(sizeof(double) * NS);
    orc_project(gi, gd, ang, f, t);
    double data = 0.0;
    for (long k = 0; k < NS; ++k) data += w[k] * (t[k] - y[k]) * (t[k] - y[k]);
    free(t);
    return data;
}

/* ------------------------------------------------------------------------ */
/* Initial image (TNLM algorithm box, step 1): filtered backprojection of    */
/* the projections of all N phases together, for the equiangular arc        */
/* detector.  The paper does not name the filter; this is the textbook       */
/* equiangular fan-beam FBP with the unwindowed discrete ramp kernel:        */
/*   R'(g_k)  = R(g_k) * sid * cos(g_k)                                     */
/*   Q(g_n)   = dg * sum_k R'(g_k) c(n - k),                                 */
/*              c(0) = 1/(8 dg^2), c(even) = 0, c(odd n) = -1/(2 pi^2 sin^2(n dg)) */
/*   f(x)     = sum_views dbeta * Q(g'(x)) / L(x)^2,  dbeta = 2 pi / (N V)   */
/* with g'(x) the fan angle of x, L its distance to the source, and Q read   */
/* by linear interpolation (zero beyond the detector).  Every phase of the   */
/* output receives the same image.                                          */
/* ------------------------------------------------------------------------ */
void orc_fbp(const int* gi, const double* gd, const double* ang, const double* y, double* f)
{
    const int B = NB;
    const long M = (long)NPH * NV;
    const double dg = BINW / SDD;
    const double dbeta = 2.0 * ORC_PI / (double)M;
    const long npx = (long)NX * NY;
    double* Q = (double*)malloc(sizeof(double) * M * B);
    double* c = (double*)malloc(sizeof(double) * (2 * B - 1));
    for (int n = -(B - 1); n <= B - 1; ++n) {
        double v;
        if (n == 0) v = 1.0 / (8.0 * dg * dg);
        else if (n % 2 == 0) v = 0.0;
        else {
            double s = sin(n * dg);
            v = -1.0 / (2.0 * ORC_PI * ORC_PI * s * s);
        }
        c[n + B - 1] = v;
    }
#pragma omp parallel for schedule(static)
    for (long v = 0; v < M; ++v) {
        for (int n = 0; n < B; ++n) {
            double acc = 0.0;
            for (int k = 0; k < B; ++k) {
                double gk = ((double)k - 0.5 * (B - 1)) * dg;
                acc += y[v * B + k] * SID * cos(gk) * c[n - k + B - 1];
            }
            Q[v * B + n] = dg * acc;
        }
    }
#pragma omp parallel for schedule(static)
    for (long p = 0; p < npx; ++p) {
        int ix = (int)(p % NX), iy = (int)(p / NX);
        double px_ = ((double)ix - 0.5 * (NX - 1)) * PIX;
        double py_ = ((double)iy - 0.5 * (NY - 1)) * PIX;
        double acc = 0.0;
        for (long v = 0; v < M; ++v) {
            double th = ang[v];
            double sx = SID * cos(th), sy = SID * sin(th);
            double cx = -cos(th), cy = -sin(th);           /* central ray */
            double dx = px_ - sx, dy = py_ - sy;
            double along = cx * dx + cy * dy;               /* dot(c, p - S) */
            double across = cx * dy - cy * dx;              /* cross(c, p - S) */
            double gam = atan2(across, along);
            double u = gam / dg + 0.5 * (B - 1);
            int k0 = (int)floor(u);
            double t = u - k0;
            double q = 0.0;
            if (k0 >= 0 && k0 < B) q += (1.0 - t) * Q[v * B + k0];
            if (k0 + 1 >= 0 && k0 + 1 < B) q += t * Q[v * B + k0 + 1];
            acc += q / (dx * dx + dy * dy);
        }
        acc *= dbeta;
        for (int i = 0; i < NPH; ++i) f[(long)i * npx + p] = acc;
    }
    free(Q);
    free(c);
}
