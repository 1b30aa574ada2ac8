/*
 * FP64 CPU oracle for the PYRO-NN known-operator CT layers (Syben et al.,
 * "PYRO-NN: Python Reconstruction Operators in Neural Networks", 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA library: every formula below is written out again from the paper
 * and from the textbook definitions the paper cites (Kak & Slaney for the
 * filters and the cosine weights, Parker for the short-scan weights,
 * Feldkamp et al. for FDK).
 *
 * Everything is plain loops in double precision, in the order the method
 * states them, so that a reader can check each function against the paper.
 * OpenMP only parallelises loops whose iterations are independent (one ray,
 * one voxel or one detector row per iteration); the scatter adjoints run
 * serially so that their result does not depend on the thread count.
 *
 * Conventions (the paper gives none; these are the readings used throughout):
 *   volume  [nz][ny][nx], x fastest; voxel centre X_i = (i - (N-1)/2) * s,
 *           i.e. the volume is centred on the iso-centre (world origin).
 *   2D sino [n_views][nu]; 3D sino [n_views][nv][nu], u fastest;
 *           detector coordinate u_k = (k - (nu-1)/2) * su (likewise v).
 *   view j: central-ray vector c = (cos b, sin b[, 0]), detector axis
 *           e_u = (-sin b, cos b[, 0]), e_v = (0, 0, 1);
 *           fan/cone source S = -SID * c, flat detector through
 *           (SDD - SID) * c, perpendicular to c.
 *   cone:   P = K [R | -R S], R = [e_u; e_v; c],
 *           K = [[SDD/su, 0, (nu-1)/2], [0, SDD/sv, (nv-1)/2], [0, 0, 1]],
 *           (x, y, w) = P (X, 1), detector index (x/w, y/w), w = depth.
 *   interpolation: bi-/trilinear in index space over the ZERO-EXTENDED
 *           array (values outside [0, N-1] are 0), i.e. the border mode of
 *           a CUDA texture.
 *   FP samples: on equally spaced planes of depth along the view's
 *           principal axis (see the forward-projection section).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define IDX2(j, i, nx) ((size_t)(j) * (size_t)(nx) + (size_t)(i))
#define IDX3(k, j, i, ny, nx) (((size_t)(k) * (size_t)(ny) + (size_t)(j)) * (size_t)(nx) + (size_t)(i))

/* ------------------------------------------------------------------------ */
/* Interpolation of zero-extended arrays                                    */
/* ------------------------------------------------------------------------ */

/* linear interpolation of a zero-extended row y[0..n-1] at index position f */
static double lerp_row(const double *y, int n, double f)
{
    double f0 = floor(f);
    double a = f - f0;
    long i0 = (long)f0;
    double v = 0.0;
    if (i0 >= 0 && i0 < n) v += (1.0 - a) * y[i0];
    if (i0 + 1 >= 0 && i0 + 1 < n) v += a * y[i0 + 1];
    return v;
}

/* bilinear interpolation of a zero-extended image img[ny][nx] at (fx, fy) */
static double interp2(const double *img, int nx, int ny, double fx, double fy)
{
    double x0 = floor(fx), y0 = floor(fy);
    double ax = fx - x0, ay = fy - y0;
    double v = 0.0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            long i = (long)x0 + dx, j = (long)y0 + dy;
            if (i < 0 || i >= nx || j < 0 || j >= ny) continue;
            double w = (dx ? ax : 1.0 - ax) * (dy ? ay : 1.0 - ay);
            v += w * img[IDX2(j, i, nx)];
        }
    return v;
}

/* transpose of interp2: add val * weight into the four neighbours */
static void scatter2(double *img, int nx, int ny, double fx, double fy, double val)
{
    double x0 = floor(fx), y0 = floor(fy);
    double ax = fx - x0, ay = fy - y0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            long i = (long)x0 + dx, j = (long)y0 + dy;
            if (i < 0 || i >= nx || j < 0 || j >= ny) continue;
            double w = (dx ? ax : 1.0 - ax) * (dy ? ay : 1.0 - ay);
            img[IDX2(j, i, nx)] += w * val;
        }
}

/* trilinear interpolation of a zero-extended volume vol[nz][ny][nx] */
static double interp3(const double *vol, int nx, int ny, int nz, double fx, double fy, double fz)
{
    double x0 = floor(fx), y0 = floor(fy), z0 = floor(fz);
    double ax = fx - x0, ay = fy - y0, az = fz - z0;
    double v = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                long i = (long)x0 + dx, j = (long)y0 + dy, k = (long)z0 + dz;
                if (i < 0 || i >= nx || j < 0 || j >= ny || k < 0 || k >= nz) continue;
                double w = (dx ? ax : 1.0 - ax) * (dy ? ay : 1.0 - ay) * (dz ? az : 1.0 - az);
                v += w * vol[IDX3(k, j, i, ny, nx)];
            }
    return v;
}

/* transpose of interp3 */
static void scatter3(double *vol, int nx, int ny, int nz, double fx, double fy, double fz, double val)
{
    double x0 = floor(fx), y0 = floor(fy), z0 = floor(fz);
    double ax = fx - x0, ay = fy - y0, az = fz - z0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                long i = (long)x0 + dx, j = (long)y0 + dy, k = (long)z0 + dz;
                if (i < 0 || i >= nx || j < 0 || j >= ny || k < 0 || k >= nz) continue;
                double w = (dx ? ax : 1.0 - ax) * (dy ? ay : 1.0 - ay) * (dz ? az : 1.0 - az);
                vol[IDX3(k, j, i, ny, nx)] += w * val;
            }
}

/* ------------------------------------------------------------------------ */
/* Geometry (Section "Reconstruction & Geometry", "Trajectories")           */
/* ------------------------------------------------------------------------ */

/* Circular cone-beam trajectory as projection matrices P = K [R | -R S]. */
void oracle_circular_pmats(int n_views, const double *angles, double sid, double sdd,
                           int nu, int nv, double su, double sv, double *P)
{
    for (int j = 0; j < n_views; ++j) {
        double b = angles[j];
        double c[3] = {cos(b), sin(b), 0.0};
        double eu[3] = {-sin(b), cos(b), 0.0};
        double ev[3] = {0.0, 0.0, 1.0};
        double S[3] = {-sid * c[0], -sid * c[1], -sid * c[2]};
        double R[3][3], t[3];
        for (int a = 0; a < 3; ++a) {
            R[0][a] = eu[a];
            R[1][a] = ev[a];
            R[2][a] = c[a];
        }
        for (int r = 0; r < 3; ++r) t[r] = -(R[r][0] * S[0] + R[r][1] * S[1] + R[r][2] * S[2]);
        double K[3][3] = {{sdd / su, 0.0, 0.5 * (nu - 1)}, {0.0, sdd / sv, 0.5 * (nv - 1)}, {0.0, 0.0, 1.0}};
        double *Pj = P + 12 * (size_t)j;
        for (int r = 0; r < 3; ++r) {
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int q = 0; q < 3; ++q) s += K[r][q] * R[q][a];
                Pj[4 * r + a] = s;
            }
            double s = 0.0;
            for (int q = 0; q < 3; ++q) s += K[r][q] * t[q];
            Pj[4 * r + 3] = s;
        }
    }
}

/* Scale a projection matrix so that its third row has a unit-norm 3-vector
 * and the iso-centre lies at positive depth; then w = depth of X along the
 * principal ray.  (x/w, y/w) is unchanged by this homogeneous rescaling. */
static void normalise_pmat(const double *Pin, double *P)
{
    double n = sqrt(Pin[8] * Pin[8] + Pin[9] * Pin[9] + Pin[10] * Pin[10]);
    double s = (Pin[11] >= 0.0 ? 1.0 : -1.0) / n;
    for (int a = 0; a < 12; ++a) P[a] = s * Pin[a];
}

/* inverse of the left 3x3 block M of P by cofactors, and source S = -M^-1 p4 */
static void pmat_inverse(const double *P, double Minv[3][3], double S[3])
{
    double m[3][3];
    for (int r = 0; r < 3; ++r)
        for (int a = 0; a < 3; ++a) m[r][a] = P[4 * r + a];
    double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                 m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                 m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    Minv[0][0] = (m[1][1] * m[2][2] - m[1][2] * m[2][1]) / det;
    Minv[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / det;
    Minv[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / det;
    Minv[1][0] = (m[1][2] * m[2][0] - m[1][0] * m[2][2]) / det;
    Minv[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / det;
    Minv[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / det;
    Minv[2][0] = (m[1][0] * m[2][1] - m[1][1] * m[2][0]) / det;
    Minv[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / det;
    Minv[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / det;
    for (int r = 0; r < 3; ++r) S[r] = -(Minv[r][0] * P[3] + Minv[r][1] * P[7] + Minv[r][2] * P[11]);
}

/* cone ray of detector pixel (k, l) of a normalised P: g = M^-1 (k, l, 1), the
 * direction with unit depth (P (S + w g, 1) = w (k, l, 1)) */
static void cone_ray(const double Minv[3][3], double k, double l, double g[3])
{
    for (int r = 0; r < 3; ++r) g[r] = Minv[r][0] * k + Minv[r][1] * l + Minv[r][2];
}

/* Half diagonal of the interpolant's support box: (N+1)*s per axis. */
static double support_radius3(int nx, int ny, int nz, double sx, double sy, double sz)
{
    double a = (nx + 1) * sx, b = (ny + 1) * sy, c = (nz + 1) * sz;
    return 0.5 * sqrt(a * a + b * b + c * c);
}

static double support_radius2(int nx, int ny, double sx, double sy)
{
    double a = (nx + 1) * sx, b = (ny + 1) * sy;
    return 0.5 * sqrt(a * a + b * b);
}

/* ------------------------------------------------------------------------ */
/* Ray-driven forward projection (Section "The Operator as a Layer")        */
/*   The ray of a detector pixel is X(w) = a + w g, parametrised by the     */
/*   depth w along the view's principal axis (g has unit depth component).  */
/*   Samples lie on equally spaced depth planes w_m = w0 + m dt, m = -M..M, */
/*   w0 the depth of the iso-centre, M = ceil(T / dt), T the half diagonal  */
/*   of the support box:  p = dt |g| sum_m f(a + w_m g)                     */
/*   (a Riemann sum of the line integral with step dt |g| along the ray).   */
/* ------------------------------------------------------------------------ */

static double line_integral2(const double *img, int nx, int ny, double sx, double sy, double dt,
                             const double a[2], const double g[2], double w0)
{
    double T = support_radius2(nx, ny, sx, sy);
    long M = (long)ceil(T / dt);
    double acc = 0.0;
    for (long m = -M; m <= M; ++m) {
        double w = w0 + (double)m * dt;
        double X = a[0] + w * g[0], Y = a[1] + w * g[1];
        acc += interp2(img, nx, ny, X / sx + 0.5 * (nx - 1), Y / sy + 0.5 * (ny - 1));
    }
    return dt * sqrt(g[0] * g[0] + g[1] * g[1]) * acc;
}

static void line_scatter2(double *img, int nx, int ny, double sx, double sy, double dt,
                          const double a[2], const double g[2], double w0, double val)
{
    double T = support_radius2(nx, ny, sx, sy);
    long M = (long)ceil(T / dt);
    double wt = dt * sqrt(g[0] * g[0] + g[1] * g[1]) * val;
    for (long m = -M; m <= M; ++m) {
        double w = w0 + (double)m * dt;
        double X = a[0] + w * g[0], Y = a[1] + w * g[1];
        scatter2(img, nx, ny, X / sx + 0.5 * (nx - 1), Y / sy + 0.5 * (ny - 1), wt);
    }
}

static double line_integral3(const double *vol, int nx, int ny, int nz, double sx, double sy, double sz,
                             double dt, const double a[3], const double g[3], double w0)
{
    double T = support_radius3(nx, ny, nz, sx, sy, sz);
    long M = (long)ceil(T / dt);
    double acc = 0.0;
    for (long m = -M; m <= M; ++m) {
        double w = w0 + (double)m * dt;
        double X = a[0] + w * g[0], Y = a[1] + w * g[1], Z = a[2] + w * g[2];
        acc += interp3(vol, nx, ny, nz, X / sx + 0.5 * (nx - 1), Y / sy + 0.5 * (ny - 1), Z / sz + 0.5 * (nz - 1));
    }
    return dt * sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) * acc;
}

static void line_scatter3(double *vol, int nx, int ny, int nz, double sx, double sy, double sz, double dt,
                          const double a[3], const double g[3], double w0, double val)
{
    double T = support_radius3(nx, ny, nz, sx, sy, sz);
    long M = (long)ceil(T / dt);
    double wt = dt * sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) * val;
    for (long m = -M; m <= M; ++m) {
        double w = w0 + (double)m * dt;
        double X = a[0] + w * g[0], Y = a[1] + w * g[1], Z = a[2] + w * g[2];
        scatter3(vol, nx, ny, nz, X / sx + 0.5 * (nx - 1), Y / sy + 0.5 * (ny - 1), Z / sz + 0.5 * (nz - 1), wt);
    }
}

/* ray of bin k of a 2D view: parallel beam a = u e_u, g = c, w0 = 0;
 * fan beam a = S = -SID c, g = c + (u / SDD) e_u (unit depth), w0 = SID */
static void ray2d(int fan, double beta, double sid, double sdd, int nu, double su, int k, double a[2], double g[2],
                  double *w0)
{
    double c[2] = {cos(beta), sin(beta)};
    double eu[2] = {-sin(beta), cos(beta)};
    double u = (k - 0.5 * (nu - 1)) * su;
    if (!fan) {
        a[0] = u * eu[0];
        a[1] = u * eu[1];
        g[0] = c[0];
        g[1] = c[1];
        *w0 = 0.0;
    } else {
        a[0] = -sid * c[0];
        a[1] = -sid * c[1];
        g[0] = c[0] + (u / sdd) * eu[0];
        g[1] = c[1] + (u / sdd) * eu[1];
        *w0 = sid;
    }
}

static void fp2d(int fan, const double *img, int nx, int ny, double sx, double sy, int nu, double su,
                 int n_views, const double *angles, double sid, double sdd, double dt, double *sino)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < n_views; ++j)
        for (int k = 0; k < nu; ++k) {
            double a[2], g[2], w0;
            ray2d(fan, angles[j], sid, sdd, nu, su, k, a, g, &w0);
            sino[IDX2(j, k, nu)] = line_integral2(img, nx, ny, sx, sy, dt, a, g, w0);
        }
}

static void fp2d_adjoint(int fan, const double *sino, int nx, int ny, double sx, double sy, int nu, double su,
                         int n_views, const double *angles, double sid, double sdd, double dt, double *img)
{
    memset(img, 0, sizeof(double) * (size_t)nx * ny);
    for (int j = 0; j < n_views; ++j)
        for (int k = 0; k < nu; ++k) {
            double a[2], g[2], w0;
            ray2d(fan, angles[j], sid, sdd, nu, su, k, a, g, &w0);
            line_scatter2(img, nx, ny, sx, sy, dt, a, g, w0, sino[IDX2(j, k, nu)]);
        }
}

void oracle_fp_par2d(const double *img, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                     const double *angles, double dt, double *sino)
{
    fp2d(0, img, nx, ny, sx, sy, nu, su, n_views, angles, 0.0, 0.0, dt, sino);
}

void oracle_fp_fan2d(const double *img, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                     const double *angles, double sid, double sdd, double dt, double *sino)
{
    fp2d(1, img, nx, ny, sx, sy, nu, su, n_views, angles, sid, sdd, dt, sino);
}

void oracle_fpT_par2d(const double *sino, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                      const double *angles, double dt, double *img)
{
    fp2d_adjoint(0, sino, nx, ny, sx, sy, nu, su, n_views, angles, 0.0, 0.0, dt, img);
}

void oracle_fpT_fan2d(const double *sino, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                      const double *angles, double sid, double sdd, double dt, double *img)
{
    fp2d_adjoint(1, sino, nx, ny, sx, sy, nu, su, n_views, angles, sid, sdd, dt, img);
}

void oracle_fp_cone3d(const double *vol, int nx, int ny, int nz, double sx, double sy, double sz, int nu, int nv,
                      int n_views, const double *pmats, double dt, double *sino)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < n_views; ++j) {
        double Pn[12], Minv[3][3], S[3];
        normalise_pmat(pmats + 12 * (size_t)j, Pn);
        pmat_inverse(Pn, Minv, S);
        for (int l = 0; l < nv; ++l)
            for (int k = 0; k < nu; ++k) {
                double g[3];
                cone_ray(Minv, (double)k, (double)l, g);
                sino[IDX3(j, l, k, nv, nu)] = line_integral3(vol, nx, ny, nz, sx, sy, sz, dt, S, g, Pn[11]);
            }
    }
}

/* the same line integrals for an arbitrary list of (view, k, l) detector pixels */
void oracle_fp_cone3d_rays(const double *vol, int nx, int ny, int nz, double sx, double sy, double sz,
                           const double *pmats, double dt, int n_rays, const int *view, const int *kk,
                           const int *ll, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n_rays; ++r) {
        double Pn[12], Minv[3][3], S[3], g[3];
        normalise_pmat(pmats + 12 * (size_t)view[r], Pn);
        pmat_inverse(Pn, Minv, S);
        cone_ray(Minv, (double)kk[r], (double)ll[r], g);
        out[r] = line_integral3(vol, nx, ny, nz, sx, sy, sz, dt, S, g, Pn[11]);
    }
}

void oracle_fpT_cone3d(const double *sino, int nx, int ny, int nz, double sx, double sy, double sz, int nu, int nv,
                       int n_views, const double *pmats, double dt, double *vol)
{
    memset(vol, 0, sizeof(double) * (size_t)nx * ny * nz);
    for (int j = 0; j < n_views; ++j) {
        double Pn[12], Minv[3][3], S[3];
        normalise_pmat(pmats + 12 * (size_t)j, Pn);
        pmat_inverse(Pn, Minv, S);
        for (int l = 0; l < nv; ++l)
            for (int k = 0; k < nu; ++k) {
                double g[3];
                cone_ray(Minv, (double)k, (double)l, g);
                line_scatter3(vol, nx, ny, nz, sx, sy, sz, dt, S, g, Pn[11], sino[IDX3(j, l, k, nv, nu)]);
            }
    }
}

/* The exact adjoint at a list of voxels (i, j, kz), from the definition:
 * (A^T y)_v = sum over views and detector pixels (k, l) of y(k, l) dt |g|
 * sum_m t_v(S + w_m g), t_v the trilinear tent of voxel v (the weight the
 * interpolation gives v at a point).  t_v vanishes outside the box of half
 * width one voxel around v, so per view only the pixels whose ray meets that
 * box contribute: those (k, l) inside the projection of the box, which lies
 * in the bounding rectangle of its eight projected corners (positive depth);
 * along such a ray only the planes w_m inside the box's slab on every axis
 * contribute.  Every other term of the sum is zero. */
void oracle_fpT_cone3d_voxels(const double *sino, int nx, int ny, int nz, double sx, double sy, double sz, int nu,
                              int nv, int n_views, const double *pmats, double dt, int n_vox, const int *ii,
                              const int *jj, const int *kk, double *out)
{
    const double T = support_radius3(nx, ny, nz, sx, sy, sz);
    const long M = (long)ceil(T / dt);
    const double s[3] = {sx, sy, sz};
    const double half[3] = {0.5 * (nx - 1), 0.5 * (ny - 1), 0.5 * (nz - 1)};
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n_vox; ++r) {
        const int v[3] = {ii[r], jj[r], kk[r]};
        double Xv[3];
        for (int a = 0; a < 3; ++a) Xv[a] = (v[a] - half[a]) * s[a];
        double acc = 0.0;
        for (int j = 0; j < n_views; ++j) {
            double Pn[12], Minv[3][3], S[3];
            normalise_pmat(pmats + 12 * (size_t)j, Pn);
            pmat_inverse(Pn, Minv, S);
            double kmin = 1e300, kmax = -1e300, lmin = 1e300, lmax = -1e300;
            for (int c = 0; c < 8; ++c) {
                double X[3];
                for (int a = 0; a < 3; ++a) X[a] = Xv[a] + (((c >> a) & 1) ? s[a] : -s[a]);
                const double x = Pn[0] * X[0] + Pn[1] * X[1] + Pn[2] * X[2] + Pn[3];
                const double y = Pn[4] * X[0] + Pn[5] * X[1] + Pn[6] * X[2] + Pn[7];
                const double w = Pn[8] * X[0] + Pn[9] * X[1] + Pn[10] * X[2] + Pn[11];
                kmin = fmin(kmin, x / w);
                kmax = fmax(kmax, x / w);
                lmin = fmin(lmin, y / w);
                lmax = fmax(lmax, y / w);
            }
            const int k0 = (int)fmax(0.0, ceil(kmin)), k1 = (int)fmin(nu - 1.0, floor(kmax));
            const int l0 = (int)fmax(0.0, ceil(lmin)), l1 = (int)fmin(nv - 1.0, floor(lmax));
            for (int l = l0; l <= l1; ++l)
                for (int k = k0; k <= k1; ++k) {
                    const double y = sino[IDX3(j, l, k, nv, nu)];
                    if (y == 0.0) continue;
                    double g[3];
                    cone_ray(Minv, (double)k, (double)l, g);
                    /* planes whose sample lies in the box on every axis */
                    double wlo = -1e300, whi = 1e300;
                    for (int a = 0; a < 3; ++a) {
                        if (g[a] != 0.0) {
                            const double t1 = (Xv[a] - s[a] - S[a]) / g[a], t2 = (Xv[a] + s[a] - S[a]) / g[a];
                            wlo = fmax(wlo, fmin(t1, t2));
                            whi = fmin(whi, fmax(t1, t2));
                        } else if (fabs(S[a] - Xv[a]) >= s[a]) {
                            wlo = 1.0;
                            whi = -1.0;
                        }
                    }
                    const long m0 = (long)fmax((double)-M, floor((wlo - Pn[11]) / dt));
                    const long m1 = (long)fmin((double)M, ceil((whi - Pn[11]) / dt));
                    double tsum = 0.0;
                    for (long m = m0; m <= m1; ++m) {
                        const double w = Pn[11] + (double)m * dt;
                        double t = 1.0;
                        for (int a = 0; a < 3; ++a) {
                            const double d = fabs((S[a] + w * g[a]) / s[a] + half[a] - v[a]);
                            t *= d < 1.0 ? 1.0 - d : 0.0;
                        }
                        tsum += t;
                    }
                    acc += y * dt * sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) * tsum;
                }
        }
        out[r] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Voxel-driven back-projection (Section "The Operator as a Layer")         */
/*   x(X) = scale * sum_j omega_j(X) * L(y_j; k_j(X)[, l_j(X)])             */
/*   omega = (SID / L)^wexp, wexp in {0, 1, 2}, L = depth of X from source. */
/* ------------------------------------------------------------------------ */

/* detector index of pixel centre X in a 2D view and its source distance L */
static double bp2d_index(int fan, double beta, double sid, double sdd, int nu, double su, double X, double Y,
                         double *L)
{
    double c0 = cos(beta), c1 = sin(beta);
    double eu0 = -sin(beta), eu1 = cos(beta);
    double s = X * eu0 + Y * eu1; /* coordinate of X along e_u */
    if (!fan) {
        *L = 1.0;
        return s / su + 0.5 * (nu - 1);
    }
    /* X - S = X + sid c, depth along c */
    double depth = X * c0 + Y * c1 + sid;
    *L = depth;
    return sdd * s / (su * depth) + 0.5 * (nu - 1);
}

static double weight_pow(double sid, double L, int wexp)
{
    double r = sid / L;
    return wexp == 0 ? 1.0 : (wexp == 1 ? r : r * r);
}

static void bp2d(int fan, const double *sino, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                 const double *angles, double sid, double sdd, int wexp, double scale, double *img)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double X = (i - 0.5 * (nx - 1)) * sx, Y = (j - 0.5 * (ny - 1)) * sy;
            double acc = 0.0;
            for (int v = 0; v < n_views; ++v) {
                double L;
                double k = bp2d_index(fan, angles[v], sid, sdd, nu, su, X, Y, &L);
                double w = fan ? weight_pow(sid, L, wexp) : 1.0;
                acc += w * lerp_row(sino + IDX2(v, 0, nu), nu, k);
            }
            img[IDX2(j, i, nx)] = scale * acc;
        }
}

/* transpose of bp2d: scatter scale * omega * (linear weights) * g into the detector */
static void bp2d_transpose(int fan, const double *img, int nx, int ny, double sx, double sy, int nu, double su,
                           int n_views, const double *angles, double sid, double sdd, int wexp, double scale,
                           double *sino)
{
    memset(sino, 0, sizeof(double) * (size_t)n_views * nu);
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < n_views; ++v)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double X = (i - 0.5 * (nx - 1)) * sx, Y = (j - 0.5 * (ny - 1)) * sy;
                double L;
                double k = bp2d_index(fan, angles[v], sid, sdd, nu, su, X, Y, &L);
                double w = fan ? weight_pow(sid, L, wexp) : 1.0;
                double g = scale * w * img[IDX2(j, i, nx)];
                double k0 = floor(k), a = k - k0;
                long q = (long)k0;
                double *row = sino + IDX2(v, 0, nu);
                if (q >= 0 && q < nu) row[q] += (1.0 - a) * g;
                if (q + 1 >= 0 && q + 1 < nu) row[q + 1] += a * g;
            }
}

void oracle_bp_par2d(const double *sino, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                     const double *angles, double scale, double *img)
{
    bp2d(0, sino, nx, ny, sx, sy, nu, su, n_views, angles, 0.0, 0.0, 0, scale, img);
}

void oracle_bp_fan2d(const double *sino, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                     const double *angles, double sid, double sdd, int wexp, double scale, double *img)
{
    bp2d(1, sino, nx, ny, sx, sy, nu, su, n_views, angles, sid, sdd, wexp, scale, img);
}

void oracle_bpT_par2d(const double *img, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                      const double *angles, double scale, double *sino)
{
    bp2d_transpose(0, img, nx, ny, sx, sy, nu, su, n_views, angles, 0.0, 0.0, 0, scale, sino);
}

void oracle_bpT_fan2d(const double *img, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                      const double *angles, double sid, double sdd, int wexp, double scale, double *sino)
{
    bp2d_transpose(1, img, nx, ny, sx, sy, nu, su, n_views, angles, sid, sdd, wexp, scale, sino);
}

/* one voxel of the cone-beam voxel-driven back-projection */
static double bp_cone_voxel(const double *sino, int nu, int nv, int n_views, const double *pn, double X, double Y,
                            double Z, double sid, int wexp)
{
    double acc = 0.0;
    for (int v = 0; v < n_views; ++v) {
        const double *P = pn + 12 * (size_t)v;
        double x = P[0] * X + P[1] * Y + P[2] * Z + P[3];
        double y = P[4] * X + P[5] * Y + P[6] * Z + P[7];
        double w = P[8] * X + P[9] * Y + P[10] * Z + P[11];
        double k = x / w, l = y / w;
        acc += weight_pow(sid, w, wexp) * interp2(sino + IDX3(v, 0, 0, nv, nu), nu, nv, k, l);
    }
    return acc;
}

static double *normalised_pmats(int n_views, const double *pmats)
{
    double *pn = (double *)malloc(sizeof(double) * 12 * (size_t)n_views);
    for (int v = 0; v < n_views; ++v) normalise_pmat(pmats + 12 * (size_t)v, pn + 12 * (size_t)v);
    return pn;
}

void oracle_bp_cone3d(const double *sino, int nx, int ny, int nz, double sx, double sy, double sz, int nu, int nv,
                      int n_views, const double *pmats, double sid, int wexp, double scale, double *vol)
{
    double *pn = normalised_pmats(n_views, pmats);
#pragma omp parallel for schedule(dynamic, 1)
    for (int kz = 0; kz < nz; ++kz)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double X = (i - 0.5 * (nx - 1)) * sx, Y = (j - 0.5 * (ny - 1)) * sy, Z = (kz - 0.5 * (nz - 1)) * sz;
                vol[IDX3(kz, j, i, ny, nx)] = scale * bp_cone_voxel(sino, nu, nv, n_views, pn, X, Y, Z, sid, wexp);
            }
    free(pn);
}

/* the same back-projection for an arbitrary list of voxels (i, j, kz) */
void oracle_bp_cone3d_voxels(const double *sino, int nx, int ny, int nz, double sx, double sy, double sz, int nu,
                             int nv, int n_views, const double *pmats, double sid, int wexp, double scale, int n_vox,
                             const int *ii, const int *jj, const int *kk, double *out)
{
    double *pn = normalised_pmats(n_views, pmats);
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < n_vox; ++r) {
        double X = (ii[r] - 0.5 * (nx - 1)) * sx, Y = (jj[r] - 0.5 * (ny - 1)) * sy, Z = (kk[r] - 0.5 * (nz - 1)) * sz;
        out[r] = scale * bp_cone_voxel(sino, nu, nv, n_views, pn, X, Y, Z, sid, wexp);
    }
    free(pn);
}

void oracle_bpT_cone3d(const double *vol, int nx, int ny, int nz, double sx, double sy, double sz, int nu, int nv,
                       int n_views, const double *pmats, double sid, int wexp, double scale, double *sino)
{
    double *pn = normalised_pmats(n_views, pmats);
    memset(sino, 0, sizeof(double) * (size_t)n_views * nu * nv);
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < n_views; ++v) {
        const double *P = pn + 12 * (size_t)v;
        for (int kz = 0; kz < nz; ++kz)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double X = (i - 0.5 * (nx - 1)) * sx, Y = (j - 0.5 * (ny - 1)) * sy,
                           Z = (kz - 0.5 * (nz - 1)) * sz;
                    double x = P[0] * X + P[1] * Y + P[2] * Z + P[3];
                    double y = P[4] * X + P[5] * Y + P[6] * Z + P[7];
                    double w = P[8] * X + P[9] * Y + P[10] * Z + P[11];
                    double g = scale * weight_pow(sid, w, wexp) * vol[IDX3(kz, j, i, ny, nx)];
                    scatter2(sino + IDX3(v, 0, 0, nv, nu), nu, nv, x / w, y / w, g);
                }
    }
    free(pn);
}

/* ------------------------------------------------------------------------ */
/* Geometric correction weights (Section "Geometric Correction Weights")    */
/* ------------------------------------------------------------------------ */

/* cosine weight of detector point (u, v) in mm: SDD / sqrt(SDD^2 + u^2 + v^2) */
static double cosine_weight(double sdd, double u, double v)
{
    return sdd / sqrt(sdd * sdd + u * u + v * v);
}

/* Parker short-scan weight for view angle beta (measured from the first view)
 * and fan angle gamma, with half fan angle delta. */
double oracle_parker_weight(double beta, double gamma, double delta)
{
    if (beta < 0.0) return 0.0;
    if (beta <= 2.0 * (delta - gamma)) {
        double s = sin(0.25 * M_PI * beta / (delta - gamma));
        return s * s;
    }
    if (beta <= M_PI - 2.0 * gamma) return 1.0;
    if (beta <= M_PI + 2.0 * delta) {
        double s = sin(0.25 * M_PI * (M_PI + 2.0 * delta - beta) / (delta + gamma));
        return s * s;
    }
    return 0.0;
}

/* Redundancy weight for a scan over [0, range], 0 < range <= 2 pi (short,
 * super-short and over-scans; Section "Geometric Correction Weights" names
 * short and super-short scans).  With the volume's conventions the line of
 * ray (beta, gamma) is measured again by the ray (beta + pi + 2 gamma, -gamma)
 * (a later partner) or (beta - pi + 2 gamma, -gamma) (an earlier one).  A ray
 * with no partner inside the scan keeps weight 1.  A ray with a later partner
 * lies in the overlap at the scan start, beta in [0, range - pi - 2 gamma];
 * it takes sin^2 of a quarter period scaled to that overlap, and its partner,
 * in the overlap at the scan end, the complementary cos^2, so each line's
 * weights add to 1.  For range = pi + 2 delta this is Parker's weighting. */
double oracle_scan_weight(double beta, double gamma, double range)
{
    if (beta < 0.0 || beta > range) return 0.0;
    double later = beta + M_PI + 2.0 * gamma, earlier = beta - M_PI + 2.0 * gamma;
    double lead = range - M_PI - 2.0 * gamma;   /* overlap length at the start for this gamma */
    double trail = range - M_PI + 2.0 * gamma;  /* overlap length at the end */
    if (later <= range && lead > 0.0) {
        double s = sin(0.5 * M_PI * beta / lead);
        return s * s;
    }
    if (earlier >= 0.0 && trail > 0.0) {
        double s = sin(0.5 * M_PI * (range - beta) / trail);
        return s * s;
    }
    return 1.0;
}

static double redundancy_weight(int redund, double beta, double gamma, double delta, double range)
{
    switch (redund) {
    case 0: return 0.5;
    case 1: return oracle_parker_weight(beta, gamma, delta);
    case 3: return oracle_scan_weight(beta, gamma, range);
    default: return 1.0;
    }
}

/* p <- W_red W_cos p over a [n_views][nv][nu] sinogram (nv = 1 for fan beam).
 * cosine: apply W_cos; redund: 0 full scan (1/2), 1 Parker, 2 none (1),
 * 3 the weighting for a scan over [0, range] (oracle_scan_weight). */
void oracle_weights(double *sino, int n_views, int nv, int nu, double su, double sv, const double *angles,
                    double sdd, int cosine, int redund, double range)
{
    double delta = atan(0.5 * nu * su / sdd);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n_views; ++j)
        for (int l = 0; l < nv; ++l)
            for (int k = 0; k < nu; ++k) {
                double u = (k - 0.5 * (nu - 1)) * su;
                double v = (l - 0.5 * (nv - 1)) * sv;
                double w = 1.0;
                if (cosine) w *= cosine_weight(sdd, u, v);
                w *= redundancy_weight(redund, angles[j] - angles[0], atan(u / sdd), delta, range);
                sino[IDX3(j, l, k, nv, nu)] *= w;
            }
}

/* ------------------------------------------------------------------------ */
/* Reconstruction filters (Section "Filters", Eq. 4: F^H K F)                */
/* ------------------------------------------------------------------------ */

/* spatial Ram-Lak kernel on sample spacing tau (Kak & Slaney) */
static double ramlak_tap(long n, double tau)
{
    if (n == 0) return 1.0 / (4.0 * tau * tau);
    if (n % 2 == 0) return 0.0;
    return -1.0 / ((double)n * (double)n * M_PI * M_PI * tau * tau);
}

/* spatial Shepp-Logan kernel on sample spacing tau */
static double shepplogan_tap(long n, double tau)
{
    return -2.0 / (M_PI * M_PI * tau * tau * (4.0 * (double)n * (double)n - 1.0));
}

/* smallest power of two >= 2 nu */
int oracle_pad_length(int nu)
{
    int p = 1;
    while (p < 2 * nu) p <<= 1;
    return p;
}

/* Row filtering.  kind 0 Ram-Lak, 2 Shepp-Logan: linear convolution
 *   q[k] = tau * sum_{j=0}^{nu-1} h(k - j) p[j]
 * (equal, bin for bin, to F^H K F with K the DFT of tau*h on pn >= 2 nu).
 * kind 1 ramp, 3 custom: K given in the Fourier domain on pn points,
 *   q = crop(F^H (K . F zeropad(p))),
 * evaluated with a naive DFT; ramp K[m] = |m| / (pn tau); custom K = Kc[0..pn/2]. */
void oracle_filter_rows(const double *in, double *out, long n_rows, int nu, double tau, int kind, const double *Kc)
{
    if (kind == 0 || kind == 2) {
        double *h = (double *)malloc(sizeof(double) * (2 * (size_t)nu - 1));
        for (long n = -(nu - 1); n <= nu - 1; ++n)
            h[n + nu - 1] = kind == 0 ? ramlak_tap(n, tau) : shepplogan_tap(n, tau);
#pragma omp parallel for schedule(static)
        for (long r = 0; r < n_rows; ++r) {
            const double *p = in + (size_t)r * nu;
            double *q = out + (size_t)r * nu;
            for (int k = 0; k < nu; ++k) {
                double s = 0.0;
                for (int j = 0; j < nu; ++j) s += h[k - j + nu - 1] * p[j];
                q[k] = tau * s;
            }
        }
        free(h);
        return;
    }
    int pn = oracle_pad_length(nu);
    double *K = (double *)malloc(sizeof(double) * pn);
    for (int m = 0; m < pn; ++m) {
        int mm = m <= pn / 2 ? m : pn - m; /* K is even: K[m] = K[pn - m] */
        K[m] = kind == 1 ? (double)mm / (pn * tau) : Kc[mm];
    }
    /* twiddles e^{-2 pi i m j / pn} via exact integer reduction of m*j mod pn */
    double *cs = (double *)malloc(sizeof(double) * pn), *sn = (double *)malloc(sizeof(double) * pn);
    for (int t = 0; t < pn; ++t) {
        cs[t] = cos(2.0 * M_PI * t / pn);
        sn[t] = sin(2.0 * M_PI * t / pn);
    }
#pragma omp parallel for schedule(static)
    for (long r = 0; r < n_rows; ++r) {
        const double *p = in + (size_t)r * nu;
        double *re = (double *)malloc(sizeof(double) * pn), *im = (double *)malloc(sizeof(double) * pn);
        for (int m = 0; m < pn; ++m) { /* F: forward DFT of the zero-padded row */
            double a = 0.0, b = 0.0;
            for (int j = 0; j < nu; ++j) {
                int t = (int)(((long)m * j) % pn);
                a += p[j] * cs[t];
                b -= p[j] * sn[t];
            }
            re[m] = K[m] * a; /* K: diagonal multiplication */
            im[m] = K[m] * b;
        }
        for (int k = 0; k < nu; ++k) { /* F^H: inverse DFT, first nu bins only */
            double a = 0.0;
            for (int m = 0; m < pn; ++m) {
                int t = (int)(((long)m * k) % pn);
                a += re[m] * cs[t] - im[m] * sn[t];
            }
            out[(size_t)r * nu + k] = a / pn;
        }
        free(re);
        free(im);
    }
    free(K);
    free(cs);
    free(sn);
}

/* Gradient of a scalar loss with respect to the diagonal filter K (Eq. 6):
 * given rows p (the filter's input) and g = dL/dq (the gradient on its
 * output), dK[m] = sum_rows c_m / pn * Re( P[m] conj(G[m]) ) with P, G the
 * length-pn DFTs of the zero-padded rows and c_m = 1 for m = 0 and m = pn/2,
 * 2 otherwise (K[m] and K[pn-m] are one parameter). */
void oracle_filter_grad_K(const double *p, const double *g, long n_rows, int nu, double *dK)
{
    int pn = oracle_pad_length(nu);
    int nk = pn / 2 + 1;
    for (int m = 0; m < nk; ++m) dK[m] = 0.0;
    double *cs = (double *)malloc(sizeof(double) * pn), *sn = (double *)malloc(sizeof(double) * pn);
    for (int t = 0; t < pn; ++t) {
        cs[t] = cos(2.0 * M_PI * t / pn);
        sn[t] = sin(2.0 * M_PI * t / pn);
    }
    for (long r = 0; r < n_rows; ++r) {
        const double *pr = p + (size_t)r * nu, *gr = g + (size_t)r * nu;
        for (int m = 0; m < nk; ++m) {
            double pa = 0, pb = 0, ga = 0, gb = 0;
            for (int j = 0; j < nu; ++j) {
                int t = (int)(((long)m * j) % pn);
                pa += pr[j] * cs[t];
                pb -= pr[j] * sn[t];
                ga += gr[j] * cs[t];
                gb -= gr[j] * sn[t];
            }
            double c = (m == 0 || m == pn / 2) ? 1.0 : 2.0;
            dK[m] += c / pn * (pa * ga + pb * gb);
        }
    }
    free(cs);
    free(sn);
}

/* ------------------------------------------------------------------------ */
/* FBP / FDK (Eq. 4, Eq. 5): x = A^T F^H K F W_red W_cos p                  */
/* ------------------------------------------------------------------------ */

/* Parallel-beam FBP: Ram-Lak-type filter on spacing su, then
 * x = (pi / n_views) * sum_j L(q_j; k_j(X)). */
void oracle_fbp_par2d(const double *sino, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                      const double *angles, int kind, const double *Kc, double *img)
{
    double *q = (double *)malloc(sizeof(double) * (size_t)n_views * nu);
    oracle_filter_rows(sino, q, n_views, nu, su, kind, Kc);
    oracle_bp_par2d(q, nx, ny, sx, sy, nu, su, n_views, angles, M_PI / n_views, img);
    free(q);
}

/* Fan-beam FBP for a flat detector: W_cos, W_red, filter on the virtual
 * detector spacing su*SID/SDD, then x = dbeta * sum_j (SID/L)^2 L(q_j; k_j). */
void oracle_fbp_fan2d(const double *sino, int nx, int ny, double sx, double sy, int nu, double su, int n_views,
                      const double *angles, double dbeta, double sid, double sdd, int kind, const double *Kc,
                      int redund, double range, double *img)
{
    size_t n = (size_t)n_views * nu;
    double *w = (double *)malloc(sizeof(double) * n), *q = (double *)malloc(sizeof(double) * n);
    memcpy(w, sino, sizeof(double) * n);
    oracle_weights(w, n_views, 1, nu, su, 0.0, angles, sdd, 1, redund, range);
    oracle_filter_rows(w, q, n_views, nu, su * sid / sdd, kind, Kc);
    oracle_bp_fan2d(q, nx, ny, sx, sy, nu, su, n_views, angles, sid, sdd, 2, dbeta, img);
    free(w);
    free(q);
}

/* Cone-beam FDK (Eq. 5) with projection matrices. */
void oracle_fdk(const double *sino, int nx, int ny, int nz, double sx, double sy, double sz, int nu, int nv,
                double su, double sv, int n_views, const double *pmats, const double *angles, double dbeta,
                double sid, double sdd, int kind, const double *Kc, int redund, double range, double *vol)
{
    size_t n = (size_t)n_views * nu * nv;
    double *w = (double *)malloc(sizeof(double) * n), *q = (double *)malloc(sizeof(double) * n);
    memcpy(w, sino, sizeof(double) * n);
    oracle_weights(w, n_views, nv, nu, su, sv, angles, sdd, 1, redund, range);
    oracle_filter_rows(w, q, (long)n_views * nv, nu, su * sid / sdd, kind, Kc);
    oracle_bp_cone3d(q, nx, ny, nz, sx, sy, sz, nu, nv, n_views, pmats, sid, 2, dbeta, vol);
    free(w);
    free(q);
}

/* FDK at a list of voxels only: the same three steps, with the weighting and
 * filtering done just for the detector rows those voxels project onto. */
void oracle_fdk_voxels(const double *sino, int nx, int ny, int nz, double sx, double sy, double sz, int nu, int nv,
                       double su, double sv, int n_views, const double *pmats, const double *angles, double dbeta,
                       double sid, double sdd, int kind, const double *Kc, int redund, double range, int n_vox,
                       const int *ii,
                       const int *jj, const int *kk, double *out)
{
    size_t n = (size_t)n_views * nu * nv;
    double *pn = normalised_pmats(n_views, pmats);
    char *need = (char *)calloc((size_t)n_views * nv, 1);
    for (int r = 0; r < n_vox; ++r) {
        double X = (ii[r] - 0.5 * (nx - 1)) * sx, Y = (jj[r] - 0.5 * (ny - 1)) * sy, Z = (kk[r] - 0.5 * (nz - 1)) * sz;
        for (int v = 0; v < n_views; ++v) {
            const double *P = pn + 12 * (size_t)v;
            double y = P[4] * X + P[5] * Y + P[6] * Z + P[7];
            double w = P[8] * X + P[9] * Y + P[10] * Z + P[11];
            long l0 = (long)floor(y / w);
            for (long l = l0; l <= l0 + 1; ++l)
                if (l >= 0 && l < nv) need[(size_t)v * nv + l] = 1;
        }
    }
    double *q = (double *)calloc(n, sizeof(double));
    double *row = (double *)malloc(sizeof(double) * nu);
    for (int v = 0; v < n_views; ++v)
        for (int l = 0; l < nv; ++l) {
            if (!need[(size_t)v * nv + l]) continue;
            memcpy(row, sino + IDX3(v, l, 0, nv, nu), sizeof(double) * nu);
            /* weights of one row: view v, detector row l */
            double delta = atan(0.5 * nu * su / sdd);
            for (int k = 0; k < nu; ++k) {
                double u = (k - 0.5 * (nu - 1)) * su, vv = (l - 0.5 * (nv - 1)) * sv;
                double w = cosine_weight(sdd, u, vv);
                w *= redundancy_weight(redund, angles[v] - angles[0], atan(u / sdd), delta, range);
                row[k] *= w;
            }
            oracle_filter_rows(row, q + IDX3(v, l, 0, nv, nu), 1, nu, su * sid / sdd, kind, Kc);
        }
    free(row);
    free(need);
    free(pn);
    oracle_bp_cone3d_voxels(q, nx, ny, nz, sx, sy, sz, nu, nv, n_views, pmats, sid, 2, dbeta, n_vox, ii, jj, kk, out);
    free(q);
}

/* ------------------------------------------------------------------------ */
/* Total variation (Eq. 7), smoothed anisotropic form                       */
/*   TV(x) = sum_axes sum_i phi(x_{i+e} - x_i),  phi(d) = sqrt(d^2+e^2) - e  */
/*   (forward differences; no term past the last index on each axis)       */
/* ------------------------------------------------------------------------ */

double oracle_tv_value(const double *x, int nx, int ny, int nz, double eps)
{
    double s = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double c = x[IDX3(k, j, i, ny, nx)];
                if (i + 1 < nx) {
                    double d = x[IDX3(k, j, i + 1, ny, nx)] - c;
                    s += sqrt(d * d + eps * eps) - eps;
                }
                if (j + 1 < ny) {
                    double d = x[IDX3(k, j + 1, i, ny, nx)] - c;
                    s += sqrt(d * d + eps * eps) - eps;
                }
                if (k + 1 < nz) {
                    double d = x[IDX3(k + 1, j, i, ny, nx)] - c;
                    s += sqrt(d * d + eps * eps) - eps;
                }
            }
    return s;
}

/* gradient of oracle_tv_value: each difference d = x_b - x_a adds
 * phi'(d) to b and subtracts it from a, phi'(d) = d / sqrt(d^2 + e^2) */
void oracle_tv_grad(const double *x, int nx, int ny, int nz, double eps, double *g)
{
    memset(g, 0, sizeof(double) * (size_t)nx * ny * nz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t a = IDX3(k, j, i, ny, nx);
                size_t nb[3];
                int ok[3] = {i + 1 < nx, j + 1 < ny, k + 1 < nz};
                nb[0] = IDX3(k, j, i + 1, ny, nx);
                nb[1] = IDX3(k, j + 1, i, ny, nx);
                nb[2] = IDX3(k + 1, j, i, ny, nx);
                for (int t = 0; t < 3; ++t) {
                    if (!ok[t]) continue;
                    double d = x[nb[t]] - x[a];
                    double dp = d / sqrt(d * d + eps * eps);
                    g[nb[t]] += dp;
                    g[a] -= dp;
                }
            }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* sets the OpenMP thread count of later calls; returns the previous one */
int oracle_set_num_threads(int n)
{
    int prev = oracle_num_threads();
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return prev;
}
