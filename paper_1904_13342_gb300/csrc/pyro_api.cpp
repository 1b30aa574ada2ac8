// Host side of the C ABI declared in include/pyro.h: argument validation,
// FP64 geometry preparation (trajectory, projection-matrix normalisation,
// RQ split for the ray set-up, voxel-to-detector maps for the
// back-projectors, filter spectra), chunking of long trajectories into
// kernel-parameter-sized pieces, and dispatch to the CUDA launchers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace pyro {

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define PYRO_CUDA(call)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(PYRO_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define PYRO_CHECK(cond, ...)                        \
    do {                                             \
        if (!(cond)) return fail(PYRO_EINVAL, __VA_ARGS__); \
    } while (0)

size_t elem_size(pyro_dtype dt)
{
    return dt == PYRO_F32 ? 4 : 2;
}

bool valid_dtype(int dt)
{
    return dt == PYRO_F32 || dt == PYRO_F16 || dt == PYRO_BF16;
}

bool pos_finite(double x)
{
    return std::isfinite(x) && x > 0.0;
}

bool aligned16(const void *p)
{
    return ((uintptr_t)p & 15u) == 0;
}

// ---------------------------------------------------------------- 2D ----
struct Geo2D {
    int nx, ny, nu, nv;
    double sx, sy, su, sid, sdd, step, range;
    std::vector<double> beta;
    bool fan;
    int M;
};

int prep2d(const pyro_geom2d *g, bool fan, Geo2D &G)
{
    PYRO_CHECK(g != nullptr, "geometry is NULL");
    PYRO_CHECK(g->nx > 0 && g->ny > 0 && g->nu > 0 && g->n_views > 0, "shapes must be positive (nx=%d ny=%d nu=%d views=%d)",
               g->nx, g->ny, g->nu, g->n_views);
    PYRO_CHECK(pos_finite(g->sx) && pos_finite(g->sy) && pos_finite(g->su), "spacings must be positive and finite");
    G.nx = g->nx;
    G.ny = g->ny;
    G.nu = g->nu;
    G.nv = 1;
    G.sx = g->sx;
    G.sy = g->sy;
    G.su = g->su;
    G.fan = fan;
    G.range = g->range;
    G.beta.resize(g->n_views);
    if (g->angles) {
        for (int j = 0; j < g->n_views; ++j) {
            PYRO_CHECK(std::isfinite(g->angles[j]), "angle %d is not finite", j);
            G.beta[j] = g->angles[j];
        }
    } else {
        PYRO_CHECK(std::isfinite(g->range) && g->range != 0.0, "angles is NULL and range is not a finite non-zero value");
        for (int j = 0; j < g->n_views; ++j) G.beta[j] = j * (g->range / g->n_views);
    }
    G.step = g->step > 0.0 ? g->step : 0.5 * std::min(g->sx, g->sy);
    PYRO_CHECK(std::isfinite(G.step), "step is not finite");
    const double T = 0.5 * std::hypot((g->nx + 1) * g->sx, (g->ny + 1) * g->sy);
    const double M = std::ceil(T / G.step);
    PYRO_CHECK(M < (1 << 28), "step too small for the image (%g samples per ray)", 2 * M + 1);
    G.M = (int)M;
    G.sid = g->sid;
    G.sdd = g->sdd;
    if (fan) {
        PYRO_CHECK(pos_finite(g->sid) && pos_finite(g->sdd) && g->sdd > g->sid, "fan beam needs 0 < SID < SDD");
        PYRO_CHECK(g->sid > T, "the source (SID=%g) must lie outside the image support (radius %g)", g->sid, T);
    }
    return PYRO_OK;
}

void fill_fp2d(const Geo2D &G, int v0, int nvw, FP2DParams &p)
{
    p.nx = G.nx;
    p.ny = G.ny;
    p.nu = G.nu;
    p.n_views = nvw;
    p.view0 = v0;
    p.views_total = (int)G.beta.size();
    p.fan = G.fan;
    p.M = G.M;
    p.su = (float)G.su;
    const double cu = 0.5 * (G.nu - 1), cx = 0.5 * (G.nx - 1), cy = 0.5 * (G.ny - 1);
    p.cu = (float)cu;
    p.sdd = (float)G.sdd;
    p.dt = (float)G.step;
    auto put = [](float &hi, float &lo, double x) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    };
    for (int v = 0; v < nvw; ++v) {
        const double b = G.beta[v0 + v], c = std::cos(b), sn = std::sin(b);
        p.dir[v] = make_float2((float)c, (float)sn);
        // u = (k - cu) su; parallel: a = u e_u, g = c; fan: t = u / SDD,
        // a = SID t e_u, g = c + t e_u; e_u = (-sin b, cos b)
        double a0x, akx, a0y, aky, g0x, gkx, g0y, gky;
        if (G.fan) {
            const double t0 = -cu * G.su / G.sdd, tk = G.su / G.sdd;
            a0x = -G.sid * t0 * sn;
            akx = -G.sid * tk * sn;
            a0y = G.sid * t0 * c;
            aky = G.sid * tk * c;
            g0x = c - t0 * sn;
            gkx = -tk * sn;
            g0y = sn + t0 * c;
            gky = tk * c;
        } else {
            a0x = cu * G.su * sn;
            akx = -G.su * sn;
            a0y = -cu * G.su * c;
            aky = G.su * c;
            g0x = c;
            gkx = 0.0;
            g0y = sn;
            gky = 0.0;
        }
        FP2DLine &h = p.ln[v], &l = p.lnlo[v];
        put(h.p0x, l.p0x, cx + a0x / G.sx);
        put(h.pkx, l.pkx, akx / G.sx);
        put(h.p0y, l.p0y, cy + a0y / G.sy);
        put(h.pky, l.pky, aky / G.sy);
        put(h.q0x, l.q0x, g0x * G.step / G.sx);
        put(h.qkx, l.qkx, gkx * G.step / G.sx);
        put(h.q0y, l.q0y, g0y * G.step / G.sy);
        put(h.qky, l.qky, gky * G.step / G.sy);
    }
}

// k(X) - cu and depth for pixel (i, j), as affine maps divided by SID (fan)
void fill_bp2d(const Geo2D &G, int v0, int nvw, int wexp, float scale, BP2DParams &p)
{
    p.nx = G.nx;
    p.ny = G.ny;
    p.nu = G.nu;
    p.n_views = nvw;
    p.view0 = v0;
    p.views_total = (int)G.beta.size();
    p.wexp = G.fan ? wexp : 0;
    p.parallel = !G.fan;
    p.cu = (float)(0.5 * (G.nu - 1));
    p.scale = scale;
    const double cx = 0.5 * (G.nx - 1), cy = 0.5 * (G.ny - 1);
    for (int v = 0; v < nvw; ++v) {
        const double b = G.beta[v0 + v];
        const double c0 = std::cos(b), c1 = std::sin(b), e0 = -std::sin(b), e1 = std::cos(b);
        // e_u . X and c . X as affine maps of (i, j)
        const double ex = e0 * G.sx, ey = e1 * G.sy, ez = -(e0 * G.sx * cx + e1 * G.sy * cy);
        const double dx = c0 * G.sx, dy = c1 * G.sy, dz = -(c0 * G.sx * cx + c1 * G.sy * cy);
        double m[6];
        if (!G.fan) {
            m[0] = ex / G.su;
            m[1] = ey / G.su;
            m[2] = ez / G.su;
            m[3] = 0.0;
            m[4] = 0.0;
            m[5] = 1.0;
        } else {
            const double f = G.sdd / (G.su * G.sid);
            m[0] = f * ex;
            m[1] = f * ey;
            m[2] = f * ez;
            m[3] = dx / G.sid;
            m[4] = dy / G.sid;
            m[5] = dz / G.sid + 1.0;
        }
        for (int a = 0; a < 6; ++a) {
            p.m[v][a] = (float)m[a];
            p.mlo[v][a] = (float)(m[a] - (double)p.m[v][a]);
        }
    }
}

// ---------------------------------------------------------------- 3D ----
struct Geo3D {
    int nx, ny, nz, nu, nv;
    double sx, sy, sz, su, sv, sid, sdd, step, range;
    std::vector<double> beta;
    std::vector<double> P;  // normalised [V][12]
    std::vector<double> S;  // source [V][3]
    int M;
    double T;
};

void inv3(const double m[9], double r[9])
{
    const double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                       m[2] * (m[3] * m[7] - m[4] * m[6]);
    r[0] = (m[4] * m[8] - m[5] * m[7]) / det;
    r[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    r[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    r[3] = (m[5] * m[6] - m[3] * m[8]) / det;
    r[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    r[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    r[6] = (m[3] * m[7] - m[4] * m[6]) / det;
    r[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    r[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

int prep3d(const pyro_geom3d *g, Geo3D &G)
{
    PYRO_CHECK(g != nullptr, "geometry is NULL");
    PYRO_CHECK(g->nx > 0 && g->ny > 0 && g->nz > 0 && g->nu > 0 && g->nv > 0 && g->n_views > 0,
               "shapes must be positive");
    PYRO_CHECK(pos_finite(g->sx) && pos_finite(g->sy) && pos_finite(g->sz) && pos_finite(g->su) && pos_finite(g->sv),
               "spacings must be positive and finite");
    G.nx = g->nx;
    G.ny = g->ny;
    G.nz = g->nz;
    G.nu = g->nu;
    G.nv = g->nv;
    G.sx = g->sx;
    G.sy = g->sy;
    G.sz = g->sz;
    G.su = g->su;
    G.sv = g->sv;
    G.sid = g->sid;
    G.sdd = g->sdd;
    G.range = g->range;
    const int V = g->n_views;
    G.beta.assign(V, 0.0);
    if (g->angles) {
        for (int j = 0; j < V; ++j) {
            PYRO_CHECK(std::isfinite(g->angles[j]), "angle %d is not finite", j);
            G.beta[j] = g->angles[j];
        }
    } else if (std::isfinite(g->range) && g->range != 0.0) {
        for (int j = 0; j < V; ++j) G.beta[j] = j * (g->range / V);
    } else {
        PYRO_CHECK(g->proj_mats != nullptr, "need projection matrices, angles or a range");
    }
    G.step = g->step > 0.0 ? g->step : 0.5 * std::min(g->sx, std::min(g->sy, g->sz));
    PYRO_CHECK(std::isfinite(G.step), "step is not finite");
    const double a = (g->nx + 1) * g->sx, b = (g->ny + 1) * g->sy, c = (g->nz + 1) * g->sz;
    G.T = 0.5 * std::sqrt(a * a + b * b + c * c);
    const double M = std::ceil(G.T / G.step);
    PYRO_CHECK(M < (1 << 28), "step too small for the volume");
    G.M = (int)M;
    G.P.resize(12 * (size_t)V);
    G.S.resize(3 * (size_t)V);
    for (int j = 0; j < V; ++j) {
        double Pj[12];
        if (g->proj_mats) {
            for (int e = 0; e < 12; ++e) {
                Pj[e] = g->proj_mats[12 * (size_t)j + e];
                PYRO_CHECK(std::isfinite(Pj[e]), "projection matrix %d has a non-finite entry", j);
            }
        } else {
            PYRO_CHECK(pos_finite(g->sid) && pos_finite(g->sdd) && g->sdd > g->sid,
                       "circular trajectory needs 0 < SID < SDD");
            const double bj = G.beta[j];
            const double cc[3] = {std::cos(bj), std::sin(bj), 0.0};
            const double eu[3] = {-std::sin(bj), std::cos(bj), 0.0};
            const double ev[3] = {0.0, 0.0, 1.0};
            const double fu = g->sdd / g->su, fv = g->sdd / g->sv;
            const double cu = 0.5 * (g->nu - 1), cv = 0.5 * (g->nv - 1);
            // P = K [R | -R S] with S = -SID c, so -R S = (0, 0, SID)
            for (int e = 0; e < 3; ++e) {
                Pj[e] = fu * eu[e] + cu * cc[e];
                Pj[4 + e] = fv * ev[e] + cv * cc[e];
                Pj[8 + e] = cc[e];
            }
            Pj[3] = cu * g->sid;
            Pj[7] = cv * g->sid;
            Pj[11] = g->sid;
        }
        // normalise: unit third row, iso-centre at positive depth
        const double n = std::sqrt(Pj[8] * Pj[8] + Pj[9] * Pj[9] + Pj[10] * Pj[10]);
        PYRO_CHECK(n > 0 && std::isfinite(n), "projection matrix %d is degenerate", j);
        const double sgn = (Pj[11] >= 0.0 ? 1.0 : -1.0) / n;
        for (int e = 0; e < 12; ++e) G.P[12 * (size_t)j + e] = sgn * Pj[e];
        const double *Q = &G.P[12 * (size_t)j];
        const double Mm[9] = {Q[0], Q[1], Q[2], Q[4], Q[5], Q[6], Q[8], Q[9], Q[10]};
        const double det = Mm[0] * (Mm[4] * Mm[8] - Mm[5] * Mm[7]) - Mm[1] * (Mm[3] * Mm[8] - Mm[5] * Mm[6]) +
                           Mm[2] * (Mm[3] * Mm[7] - Mm[4] * Mm[6]);
        PYRO_CHECK(std::isfinite(det) && std::fabs(det) > 1e-300, "projection matrix %d is singular", j);
        double Mi[9];
        inv3(Mm, Mi);
        double *S = &G.S[3 * (size_t)j];
        for (int r = 0; r < 3; ++r) S[r] = -(Mi[3 * r] * Q[3] + Mi[3 * r + 1] * Q[7] + Mi[3 * r + 2] * Q[11]);
        const double dS = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
        PYRO_CHECK(dS > G.T, "view %d: the source (distance %g) must lie outside the volume support (radius %g)", j, dS,
                   G.T);
    }
    return PYRO_OK;
}

// One view's camera in FP64 for the ray-driven projector: the RQ split
// P = K R [I | -S] of the normalised matrix, q = K^-1 (k, l, 1) scaled to
// unit depth, q_x = a0 k + a1 l + a2, q_y = b0 l + b2, the source in camera
// coordinates s = R S, W = diag(1/spacing) R^T (camera -> voxel index).
// col: the rows of a detector column share their (x, y) point (the camera's
// y axis along z and no skew; the FP64 residue of the split in those
// entries, below 1e-12, is set to exact zeros so that FP32 rows agree bit
// for bit).  dz_row: voxels in z one row step moves a sample at the far
// sampled depth.
struct CamView {
    double W[9], a0, a1, a2, b0, b2, s1, s2, s3, K00, K11;
    bool col;
    double dz_row;
};

int cam_view(const Geo3D &G, int view, CamView &c)
{
    const double inv_s[3] = {1.0 / G.sx, 1.0 / G.sy, 1.0 / G.sz};
    const double *Q = &G.P[12 * (size_t)view];
    const double *S = &G.S[3 * (size_t)view];
    const double m0[3] = {Q[0], Q[1], Q[2]}, m1[3] = {Q[4], Q[5], Q[6]}, m2[3] = {Q[8], Q[9], Q[10]};
    auto dot = [](const double *x, const double *y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    // RQ split M = K R by Gram-Schmidt from the last row (|m2| = 1 here)
    double r2[3], r1[3], r0[3], t[3];
    const double K22 = std::sqrt(dot(m2, m2));
    for (int e = 0; e < 3; ++e) r2[e] = m2[e] / K22;
    const double K12 = dot(m1, r2);
    for (int e = 0; e < 3; ++e) t[e] = m1[e] - K12 * r2[e];
    const double K11 = std::sqrt(dot(t, t));
    for (int e = 0; e < 3; ++e) r1[e] = t[e] / K11;
    const double K02 = dot(m0, r2), K01 = dot(m0, r1);
    for (int e = 0; e < 3; ++e) t[e] = m0[e] - K02 * r2[e] - K01 * r1[e];
    const double K00 = std::sqrt(dot(t, t));
    if (!(K00 > 0 && K11 > 0)) return fail(PYRO_EINVAL, "projection matrix %d has a degenerate camera", view);
    for (int e = 0; e < 3; ++e) r0[e] = t[e] / K00;
    double K01s = K01;
    c.col = std::fabs(r1[0]) < 1e-12 && std::fabs(r1[1]) < 1e-12 && std::fabs(K01) < 1e-12 * K00;
    if (c.col) {
        r1[0] = r1[1] = 0.0;
        r1[2] = r1[2] > 0 ? 1.0 : -1.0;
        K01s = 0.0;
        // then r0 and r2 lie in the xy plane up to the split's rounding
        r0[2] = 0.0;
        r2[2] = 0.0;
    }
    const double b0 = 1.0 / K11, b2 = -K12 / K11;
    c.a0 = 1.0 / K00;
    c.a1 = -K01s * b0 / K00;
    c.a2 = (-K02 - K01 * b2) / K00;
    c.b0 = b0;
    c.b2 = b2;
    (void)K22;
    c.s1 = dot(r0, S);
    c.s2 = dot(r1, S);
    c.s3 = dot(r2, S);
    c.K00 = K00;
    c.K11 = K11;
    const double *R[3] = {r0, r1, r2};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) c.W[3 * a + b] = R[b][a] * inv_s[a];
    const double w_far = -dot(r2, S) + G.M * G.step;
    c.dz_row = std::fabs(b0 * r1[2] * inv_s[2]) * w_far;
    return PYRO_OK;
}

int fill_fp3d(const Geo3D &G, int v0, int nvw, FP3DParams &p)
{
    p.nx = G.nx;
    p.ny = G.ny;
    p.nz = G.nz;
    p.nu = G.nu;
    p.nv = G.nv;
    p.n_views = nvw;
    p.view0 = v0;
    p.views_total = (int)G.beta.size();
    p.M = G.M;
    p.cx = (float)(0.5 * (G.nx - 1));
    p.cy = (float)(0.5 * (G.ny - 1));
    p.cz = (float)(0.5 * (G.nz - 1));
    p.dt = (float)G.step;
    p.dt_lo = (float)(G.step - (double)p.dt);
    p.column_shared = 1;
    p.pair_rows = 64;
    auto put = [](float &hi, float &lo, double x) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    };
    for (int v = 0; v < nvw; ++v) {
        CamView c;
        if (int e = cam_view(G, v0 + v, c)) return e;
        ConeFPView &o = p.v[v], &ol = p.vlo[v];
        put(o.a0, ol.a0, c.a0);
        put(o.a1, ol.a1, c.a1);
        put(o.a2, ol.a2, c.a2);
        put(o.b0, ol.b0, c.b0);
        put(o.b2, ol.b2, c.b2);
        put(o.s1, ol.s1, c.s1);
        put(o.s2, ol.s2, c.s2);
        put(o.s3, ol.s3, c.s3);
        for (int a = 0; a < 9; ++a) put(o.W[a], ol.W[a], c.W[a]);
        // the column kernel needs 31 row steps below 29.5 voxels over the sampled depths
        if (!c.col || !(31.0 * c.dz_row <= 29.5)) p.column_shared = 0;
        // rows whose z span stays within a 32-voxel run, for two rays per lane
        const int rows = c.dz_row > 0.0 ? (int)std::min(64.0, std::floor(29.5 / c.dz_row) + 1.0) : 64;
        p.pair_rows = std::min(p.pair_rows, rows);
    }
    // two rays per lane pay off from 40 rows per window (a row step below
    // about 0.76 voxel); below that the one-ray kernels run
    if (p.pair_rows < 40) p.pair_rows = 0;
    return PYRO_OK;
}

// The gathered adjoint's per-view maps (circular-type trajectories), from
// the same camera as the projector: the sample of ray (k, l) on plane m is
// p + m q with p = W (s1 - s3 q_x, s2 - s3 q_y, 0) + c and q = dt W (q_x, q_y,
// 1); with the camera's y axis along z, x and y depend on k only and z on l
// only.  The detector column coordinate of a voxel column is the
// projection's u = (P0 . X) / (P2 . X) in voxel-index units, its depth-plane
// coordinate ((P2 . X) - depth of the iso-centre) / dt.
//
// Row step: plane m's rows step beta(m) = B + m D voxels in z, smallest in
// magnitude at an end of the plane range; a z voxel's tent reaches at most
// floor(2 / |beta|) + 1 rows, and a lane's window, starting at a multiple of
// 4 rows, holds that many plus 3 (gather_rows: 0 when more than 32 rows).
struct GatherRows {
    double beta_min;  // smallest |beta| over the planes
    double drift;     // largest |C + D l| over the rows: z shift per plane
    int nmax, wrows;
};

int gather_rows(const Geo3D &G, const CamView &c, GatherRows &r)
{
    const double B = -c.W[7] * c.s3 * c.b0, D = G.step * c.W[7] * c.b0;
    const double C0 = G.step * (c.W[7] * c.b2 + c.W[8]);
    const double b1 = B - G.M * D, b2 = B + G.M * D;
    if (b1 * b2 <= 0.0) return PYRO_EUNSUPPORTED;  // a depth plane of the support holds the source
    r.beta_min = std::min(std::fabs(b1), std::fabs(b2));
    r.drift = std::max(std::fabs(C0), std::fabs(C0 + D * (G.nv - 1)));
    const double n = std::floor(2.0 / r.beta_min + 1e-3) + 1.0;
    r.nmax = n > 64.0 ? 64 : (int)n;
    const int w = (r.nmax + 3 + 3) / 4 * 4;
    r.wrows = w <= 32 ? w : 0;
    return PYRO_OK;
}

// Capacities of the kernel's shared tables are bounds over every tile and
// view: the support of a tile's tents is (tile + 1) voxels square;
// its diagonal, seen from the nearest depth, spans at most kmax detector
// columns, and its depth at most plmax planes; a warp's 32 z voxels (and a
// tent on either side) span at most 34 / |beta| rows, widened by the z
// drift over the planes and a window.
int fill_gather(const Geo3D &G, int v0, int nvw, int accumulate, GatherParams &g)
{
    g.nx = G.nx;
    g.ny = G.ny;
    g.nz = G.nz;
    g.nu = G.nu;
    g.nv = G.nv;
    g.n_views = nvw;
    g.view0 = v0;
    g.views_total = (int)G.beta.size();
    g.M = G.M;
    g.accumulate = accumulate;
    auto put = [](float (&hl)[2], double x) {
        hl[0] = (float)x;
        hl[1] = (float)(x - (double)hl[0]);
    };
    const double cen[3] = {0.5 * (G.nx - 1), 0.5 * (G.ny - 1), 0.5 * (G.nz - 1)};
    g.tile = gather_tile(G.nx, G.ny, G.nz);
    const double side = g.tile + 1;
    const double diag = std::sqrt(2.0) * side * std::max(G.sx, G.sy);
    double kcols = 0.0, planes = 0.0, rows = 0.0;
    int wrows = 0;
    for (int v = 0; v < nvw; ++v) {
        CamView c;
        if (int e = cam_view(G, v0 + v, c)) return e;
        if (!c.col) return fail(PYRO_EUNSUPPORTED, "the gathered adjoint needs a circular-type trajectory");
        GatherRows gr;
        if (gather_rows(G, c, gr) != PYRO_OK || gr.wrows == 0)
            return fail(PYRO_EUNSUPPORTED, "detector rows too fine (or the source inside) for the gathered adjoint");
        const double *W = c.W, dt = G.step;
        GatherView &o = g.v[v];
        // x and y: q_x = a0 k + a2 (a1 = 0 here), p_a = W[3a] (s1 - s3 q_x) + c_a, q_a = dt (W[3a] q_x + W[3a+2])
        for (int a = 0; a < 2; ++a) {
            const double w0 = W[3 * a], w2 = W[3 * a + 2];
            float(&P0)[2] = a == 0 ? o.px0 : o.py0;
            float(&Pk)[2] = a == 0 ? o.pxk : o.pyk;
            float(&Q0)[2] = a == 0 ? o.qx0 : o.qy0;
            float(&Qk)[2] = a == 0 ? o.qxk : o.qyk;
            put(P0, w0 * (c.s1 - c.s3 * c.a2) + cen[a]);
            put(Pk, -w0 * c.s3 * c.a0);
            put(Q0, dt * (w0 * c.a2 + w2));
            put(Qk, dt * w0 * c.a0);
        }
        // z: q_y = b0 l + b2, p_z = W[7] (s2 - s3 q_y) + c_z, q_z = dt (W[7] q_y + W[8])
        put(o.A, c.W[7] * (c.s2 - c.s3 * c.b2) + cen[2]);
        put(o.B, -c.W[7] * c.s3 * c.b0);
        put(o.C, dt * (c.W[7] * c.b2 + c.W[8]));
        put(o.D, dt * c.W[7] * c.b0);
        // detector column and depth plane of voxel index (x, y): the
        // normalised matrix on X = (idx - c) s
        const double *Q = &G.P[12 * (size_t)(v0 + v)];
        const double s[2] = {G.sx, G.sy};
        double U[3], Wd[3];
        for (int a = 0; a < 2; ++a) {
            U[a] = Q[a] * s[a];
            Wd[a] = Q[8 + a] * s[a];
        }
        U[2] = Q[3] - Q[0] * s[0] * cen[0] - Q[1] * s[1] * cen[1];
        Wd[2] = Q[11] - Q[8] * s[0] * cen[0] - Q[9] * s[1] * cen[1];
        o.ui = (float)U[0];
        o.uj = (float)U[1];
        o.u0 = (float)U[2];
        o.wi = (float)Wd[0];
        o.wj = (float)Wd[1];
        o.w0 = (float)Wd[2];
        o.mi = (float)(Wd[0] / dt);
        o.mj = (float)(Wd[1] / dt);
        o.mc = (float)(-(Q[8] * s[0] * cen[0] + Q[9] * s[1] * cen[1]) / dt);
        o.pad = 0.0f;
        const double w_near = std::max(Q[11] - G.T, 1e-9);  // the iso-centre's depth less the support radius
        kcols = std::max(kcols, diag * c.K00 / w_near);
        const double np = side * (std::fabs(Wd[0]) + std::fabs(Wd[1])) / dt;
        planes = std::max(planes, np);
        rows = std::max(rows, (34.0 + (np + 3.0) * gr.drift) / gr.beta_min);
        wrows = std::max(wrows, gr.wrows);
    }
    g.kmax = (int)std::ceil(kcols) + 4;
    g.plmax = (int)std::ceil(planes) + 3;
    g.wrows = wrows;
    const int rmax = ((int)std::ceil(rows) + wrows + 8 + 3) / 4 * 4;
    // staged floats per warp: at least 1024 (a few columns per fill); more
    // shared memory per block costs resident blocks, which costs more than
    // refilling the stage (256^3 / 512^3 workloads: 37.9 ms / 1.16 s with
    // 1024, 44.8 ms / 1.24 s with 2048, 59.7 ms / 1.58 s with 4096)
    g.sc = std::max(1024, rmax);
    return PYRO_OK;
}

// voxel index -> (x, y, w) / SID with rows 0 and 1 centred on the detector
void fill_bp3d(const Geo3D &G, int v0, int nvw, int wexp, float scale, int accumulate, BP3DParams &p)
{
    p.nx = G.nx;
    p.ny = G.ny;
    p.nz = G.nz;
    p.nu = G.nu;
    p.nv = G.nv;
    p.n_views = nvw;
    p.view0 = v0;
    p.views_total = (int)G.beta.size();
    p.wexp = wexp;
    p.accumulate = accumulate;
    p.cu = (float)(0.5 * (G.nu - 1));
    p.cv = (float)(0.5 * (G.nv - 1));
    p.scale = scale;
    const double cu = 0.5 * (G.nu - 1), cv = 0.5 * (G.nv - 1);
    const double c[3] = {0.5 * (G.nx - 1), 0.5 * (G.ny - 1), 0.5 * (G.nz - 1)};
    const double s[3] = {G.sx, G.sy, G.sz};
    const double wscale = G.sid > 0 ? 1.0 / G.sid : 1.0;
    int zinv = 1;
    for (int v = 0; v < nvw; ++v) {
        const double *Q = &G.P[12 * (size_t)(v0 + v)];
        double A[12];
        for (int r = 0; r < 3; ++r) {
            // P (X, 1) with X = (idx - c) s
            double off = Q[4 * r + 3];
            for (int a = 0; a < 3; ++a) {
                A[4 * r + a] = Q[4 * r + a] * s[a];
                off -= Q[4 * r + a] * s[a] * c[a];
            }
            A[4 * r + 3] = off;
        }
        for (int a = 0; a < 4; ++a) {
            A[a] -= cu * A[8 + a];
            A[4 + a] -= cv * A[8 + a];
        }
        for (int a = 0; a < 12; ++a) {
            const double x = A[a] * wscale;
            p.P[v][a] = (float)x;
            p.Plo[v][a] = (float)(x - (double)p.P[v][a]);
        }
        if (p.P[v][2] != 0.0f || p.P[v][10] != 0.0f) zinv = 0;
    }
    p.z_invariant = zinv;
}

// ------------------------------------------------------------- filters ---
int log2_exact(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

int pad_length(int nu)
{
    int p = 1;
    while (p < 2 * nu) p <<= 1;
    return p;
}

// K[m], m = 0..pn/2, of the built-in filters (FP64, cached per (kind, pn, tau))
const std::vector<float> &builtin_K(pyro_filter kind, int pn, double tau)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, double>, std::vector<float>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple((int)kind, pn, tau);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    std::vector<float> K(pn / 2 + 1);
    if (kind == PYRO_RAMP) {
        for (int m = 0; m <= pn / 2; ++m) K[m] = (float)(m / (pn * tau));
    } else {
        // taps h(n), |n| < pn/2, on the sample spacing tau (Kak & Slaney)
        std::vector<double> h(pn / 2);
        const double pi = 3.14159265358979323846;
        for (int n = 0; n < pn / 2; ++n) {
            if (kind == PYRO_RAMLAK)
                h[n] = n == 0 ? 1.0 / (4 * tau * tau) : (n % 2 ? -1.0 / ((double)n * n * pi * pi * tau * tau) : 0.0);
            else
                h[n] = -2.0 / (pi * pi * tau * tau * (4.0 * (double)n * n - 1.0));
        }
        std::vector<double> cs(pn);
        for (int t = 0; t < pn; ++t) cs[t] = std::cos(2.0 * pi * t / pn);
        for (int m = 0; m <= pn / 2; ++m) {
            double acc = h[0];
            for (int n = 1; n < pn / 2; ++n) acc += 2.0 * h[n] * cs[((long)m * n) % pn];
            K[m] = (float)(tau * acc);
        }
    }
    return cache.emplace(key, std::move(K)).first->second;
}

int fill_filter(long n_rows, int nu, double tau, pyro_filter kind, const float *custom_K, FilterParams &p)
{
    PYRO_CHECK(n_rows >= 0 && nu > 0, "n_rows must be >= 0 and nu > 0");
    PYRO_CHECK(nu <= kMaxPadLength / 2, "nu=%d exceeds the supported row length %d", nu, kMaxPadLength / 2);
    PYRO_CHECK(kind == PYRO_RAMLAK || kind == PYRO_RAMP || kind == PYRO_SHEPP_LOGAN || kind == PYRO_FILTER_CUSTOM,
               "unknown filter kind %d", (int)kind);
    if (kind == PYRO_FILTER_CUSTOM)
        PYRO_CHECK(custom_K != nullptr, "PYRO_FILTER_CUSTOM needs custom_K");
    else
        PYRO_CHECK(pos_finite(tau), "tau must be positive and finite");
    p.n_rows = n_rows;
    p.nu = nu;
    p.pn = pad_length(nu);
    p.log2pn = log2_exact(p.pn);
    p.rows_per_view = 1;
    p.n_views = 1;
    p.apply_weights = 0;
    std::memset(&p.w, 0, sizeof(p.w));
    if (kind != PYRO_FILTER_CUSTOM) {
        const std::vector<float> &K = builtin_K(kind, p.pn, tau);
        std::copy(K.begin(), K.end(), p.K);
    }
    return PYRO_OK;
}

constexpr double kPi = 3.14159265358979323846;

int fill_weights(int nu, int nv, double su, double sv, double sdd, const std::vector<double> &beta, double range,
                 int cosine, pyro_redund redund, WeightParams &w, BetaTable &bt)
{
    PYRO_CHECK(redund == PYRO_REDUND_FULL || redund == PYRO_REDUND_PARKER || redund == PYRO_REDUND_NONE ||
                   redund == PYRO_REDUND_SCAN,
               "unknown redundancy mode %d", (int)redund);
    PYRO_CHECK(pos_finite(sdd), "weights need SDD > 0");
    const int V = (int)beta.size();
    const bool by_view = redund == PYRO_REDUND_PARKER || redund == PYRO_REDUND_SCAN;
    if (by_view) PYRO_CHECK(V <= kMaxViews2D, "scan weights support at most %d views", kMaxViews2D);
    if (redund == PYRO_REDUND_SCAN)
        PYRO_CHECK(std::isfinite(range) && range > 0.0 && range <= 2.0 * kPi * (1.0 + 1e-12),
                   "PYRO_REDUND_SCAN needs 0 < range <= 2 pi (got %g)", range);
    w.nu = nu;
    w.nv = nv;
    w.n_views = V;
    w.cosine = cosine ? 1 : 0;
    w.redund = redund;
    w.su = (float)su;
    w.sv = (float)sv;
    w.cu = (float)(0.5 * (nu - 1));
    w.cv = (float)(0.5 * (nv - 1));
    w.sdd = (float)sdd;
    w.delta = redund == PYRO_REDUND_SCAN ? (float)(0.5 * (range - kPi)) : (float)std::atan(0.5 * nu * su / sdd);
    std::memset(&bt, 0, sizeof(bt));
    if (by_view)
        for (int j = 0; j < V; ++j) bt.beta[j] = (float)(beta[j] - beta[0]);
    return PYRO_OK;
}

// pointers may be NULL only when there is nothing to read or write (count == 0)
int check_io(const void *a, const void *b, long count, pyro_dtype dt)
{
    PYRO_CHECK(count >= 0, "batch / row count must be >= 0");
    if (count > 0) PYRO_CHECK(a != nullptr && b != nullptr, "input/output pointer is NULL");
    PYRO_CHECK(aligned16(a) && aligned16(b), "device pointers must be 16-byte aligned");
    PYRO_CHECK(valid_dtype(dt), "unknown dtype %d", (int)dt);
    return PYRO_OK;
}

cudaStream_t as_stream(void *s)
{
    return reinterpret_cast<cudaStream_t>(s);
}

// -------------------------------------------------------- operations ----
// work (may be NULL): a transposed copy of the batch for the staged form
int fp2d(bool fan, const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_dtype dt, void *stream,
         void *work = nullptr, size_t work_bytes = 0)
{
    if (int e = check_io(vol, sino, batch, dt)) return e;
    Geo2D G;
    if (int e = prep2d(g, fan, G)) return e;
    const size_t img = (size_t)G.nx * G.ny * elem_size(dt);
    if (work) {
        const size_t need = img * (size_t)std::max(batch, 1);
        if (work_bytes < need || !aligned16(work))
            return fail(PYRO_EWORKSPACE, "the staged 2D projector needs a 16-byte aligned workspace of %zu bytes "
                                         "(got %zu)", need, work_bytes);
    }
    if (batch == 0) return PYRO_OK;
    for (int b0 = 0; work && b0 < batch; b0 += 65535)
        PYRO_CUDA(launch_transpose2d((const char *)vol + b0 * img, (char *)work + b0 * img,
                                     std::min(65535, batch - b0), G.nx, G.ny, dt, as_stream(stream)));
    const int V = (int)G.beta.size();
    static thread_local FP2DParams p;
    for (int v0 = 0; v0 < V; v0 += kMaxViewsFP2D) {
        const int nvw = std::min(kMaxViewsFP2D, V - v0);
        fill_fp2d(G, v0, nvw, p);
        for (int b0 = 0; b0 < batch; b0 += 65535) {
            const int nb = std::min(65535, batch - b0);
            const char *vi = (const char *)vol + (size_t)b0 * img;
            const char *vt = work ? (const char *)work + (size_t)b0 * img : nullptr;
            char *so = (char *)sino + (size_t)b0 * V * G.nu * elem_size(dt);
            PYRO_CUDA(launch_fp2d(vi, vt, so, nb, p, dt, as_stream(stream)));
        }
    }
    return PYRO_OK;
}

// work (may be NULL): a transposed FP32 accumulator for the staged form
int fp2d_adjoint(bool fan, const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_dtype dt, void *stream,
                 void *work = nullptr, size_t work_bytes = 0)
{
    if (int e = check_io(sino, vol, batch, dt)) return e;
    if (dt != PYRO_F32) return fail(PYRO_EUNSUPPORTED, "the FP adjoint supports PYRO_F32 only");
    Geo2D G;
    if (int e = prep2d(g, fan, G)) return e;
    const size_t vox_bytes = sizeof(float) * (size_t)G.nx * G.ny;
    if (work) {
        const size_t need = vox_bytes * (size_t)std::max(batch, 1);
        if (work_bytes < need || !aligned16(work))
            return fail(PYRO_EWORKSPACE, "the staged 2D adjoint needs a 16-byte aligned workspace of %zu bytes "
                                         "(got %zu)", need, work_bytes);
    }
    if (batch == 0) return PYRO_OK;
    const int V = (int)G.beta.size();
    PYRO_CUDA(cudaMemsetAsync(vol, 0, vox_bytes * batch, as_stream(stream)));
    if (work) PYRO_CUDA(cudaMemsetAsync(work, 0, vox_bytes * batch, as_stream(stream)));
    static thread_local FP2DParams p;
    for (int v0 = 0; v0 < V; v0 += kMaxViewsFP2D) {
        const int nvw = std::min(kMaxViewsFP2D, V - v0);
        fill_fp2d(G, v0, nvw, p);
        for (int b0 = 0; b0 < batch; b0 += 65535) {
            const int nb = std::min(65535, batch - b0);
            const float *si = (const float *)sino + (size_t)b0 * V * G.nu;
            float *vo = (float *)vol + (size_t)b0 * G.nx * G.ny;
            float *vt = work ? (float *)work + (size_t)b0 * G.nx * G.ny : nullptr;
            PYRO_CUDA(launch_fp2d_adjoint(si, vo, vt, nb, p, as_stream(stream)));
        }
    }
    for (int b0 = 0; work && b0 < batch; b0 += 65535)
        PYRO_CUDA(launch_add_transposed((const float *)work + (size_t)b0 * G.nx * G.ny,
                                        (float *)vol + (size_t)b0 * G.nx * G.ny, std::min(65535, batch - b0), G.nx,
                                        G.ny, as_stream(stream)));
    return PYRO_OK;
}

int bp_weight_exp(pyro_bp_weight w)
{
    return w == PYRO_W_NONE ? 0 : (w == PYRO_W_INV_L ? 1 : (w == PYRO_W_INV_L2 ? 2 : -1));
}

int bp2d(bool fan, const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_bp_weight w, float scale,
         pyro_dtype sino_dt, pyro_dtype vol_dt, void *stream)
{
    if (int e = check_io(sino, vol, batch, vol_dt)) return e;
    PYRO_CHECK(valid_dtype(sino_dt), "unknown dtype");
    const int wexp = bp_weight_exp(w);
    PYRO_CHECK(wexp >= 0, "unknown back-projection weight %d", (int)w);
    PYRO_CHECK(std::isfinite(scale), "scale is not finite");
    Geo2D G;
    if (int e = prep2d(g, fan, G)) return e;
    if (batch == 0) return PYRO_OK;
    const int V = (int)G.beta.size();
    static thread_local BP2DParams p;
    for (int v0 = 0; v0 < V; v0 += kMaxViewsBP2D) {
        const int nvw = std::min(kMaxViewsBP2D, V - v0);
        fill_bp2d(G, v0, nvw, wexp, scale, p);
        for (int b0 = 0; b0 < batch; b0 += 65535) {
            const int nb = std::min(65535, batch - b0);
            const char *si = (const char *)sino + (size_t)b0 * V * G.nu * elem_size(sino_dt);
            char *vo = (char *)vol + (size_t)b0 * G.nx * G.ny * elem_size(vol_dt);
            PYRO_CUDA(launch_bp2d(si, vo, nb, p, sino_dt, vol_dt, v0 > 0, as_stream(stream)));
        }
    }
    return PYRO_OK;
}

int bp2d_transpose(bool fan, const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_bp_weight w,
                   float scale, pyro_dtype dt, void *stream)
{
    if (int e = check_io(vol, sino, batch, dt)) return e;
    if (dt != PYRO_F32) return fail(PYRO_EUNSUPPORTED, "the BP transpose supports PYRO_F32 only");
    const int wexp = bp_weight_exp(w);
    PYRO_CHECK(wexp >= 0, "unknown back-projection weight %d", (int)w);
    PYRO_CHECK(std::isfinite(scale), "scale is not finite");
    Geo2D G;
    if (int e = prep2d(g, fan, G)) return e;
    if (batch == 0) return PYRO_OK;
    const int V = (int)G.beta.size();
    PYRO_CUDA(cudaMemsetAsync(sino, 0, sizeof(float) * (size_t)batch * V * G.nu, as_stream(stream)));
    static thread_local BP2DParams p;
    for (int v0 = 0; v0 < V; v0 += kMaxViewsBP2D) {
        const int nvw = std::min(kMaxViewsBP2D, V - v0);
        fill_bp2d(G, v0, nvw, wexp, scale, p);
        for (int b0 = 0; b0 < batch; b0 += 65535) {
            const int nb = std::min(65535, batch - b0);
            const float *vi = (const float *)vol + (size_t)b0 * G.nx * G.ny;
            float *so = (float *)sino + (size_t)b0 * V * G.nu;
            PYRO_CUDA(launch_bp2d_transpose(vi, so, nb, p, as_stream(stream)));
        }
    }
    return PYRO_OK;
}

int fp3d(const void *vol, void *sino, int batch, const pyro_geom3d *g, pyro_dtype dt, bool adjoint, void *stream)
{
    if (int e = check_io(vol, sino, batch, dt)) return e;
    if (adjoint && dt != PYRO_F32) return fail(PYRO_EUNSUPPORTED, "the FP adjoint supports PYRO_F32 only");
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    if (batch == 0) return PYRO_OK;
    const int V = (int)G.beta.size();
    const size_t vox = (size_t)G.nx * G.ny * G.nz, det = (size_t)G.nu * G.nv;
    // for the adjoint `vol` is the sinogram and `sino` the output volume
    if (adjoint) PYRO_CUDA(cudaMemsetAsync(sino, 0, sizeof(float) * batch * vox, as_stream(stream)));
    static thread_local FP3DParams p;
    for (int v0 = 0; v0 < V; v0 += kMaxViewsConeFP) {
        const int nvw = std::min(kMaxViewsConeFP, V - v0);
        if (int e = fill_fp3d(G, v0, nvw, p)) return e;
        const int bstep = std::max(1, 65535 / nvw);
        for (int b0 = 0; b0 < batch; b0 += bstep) {
            const int nb = std::min(bstep, batch - b0);
            if (!adjoint) {
                const char *vi = (const char *)vol + b0 * vox * elem_size(dt);
                char *so = (char *)sino + b0 * V * det * elem_size(dt);
                PYRO_CUDA(launch_fp3d(vi, so, nb, p, dt, as_stream(stream)));
            } else {
                const float *si = (const float *)vol + b0 * V * det;
                float *vo = (float *)sino + b0 * vox;
                PYRO_CUDA(launch_fp3d_adjoint(si, vo, nb, p, as_stream(stream)));
            }
        }
    }
    return PYRO_OK;
}

// The column-shared kernels (padded z-major copy) serve a geometry when every
// view allows them and the padded copy is int-indexable.
int column_path(const Geo3D &G, FP3DParams &p, bool &column)
{
    const size_t cells = fp_padded_cells(G.nx, G.ny, G.nz);
    const int V = (int)G.beta.size();
    column = cells < (size_t)INT32_MAX;  // cell indices are ints
    for (int v0 = 0; v0 < V && column; v0 += kMaxViewsConeFP) {
        if (int e = fill_fp3d(G, v0, std::min(kMaxViewsConeFP, V - v0), p)) return e;
        column = p.column_shared != 0;
    }
    return PYRO_OK;
}

// staged cone FP: per batch item, a z-major copy of the volume in `work`,
// held in `storage` (the volume's type, or FP16 / BF16 for an FP32 volume)
int fp3d_staged(const void *vol, void *sino, int batch, const pyro_geom3d *g, void *work, size_t work_bytes,
                pyro_dtype dt, pyro_dtype storage, void *stream)
{
    if (int e = check_io(vol, sino, batch, dt)) return e;
    PYRO_CHECK(valid_dtype(storage), "unknown storage dtype %d", (int)storage);
    if (storage != dt && dt != PYRO_F32)
        return fail(PYRO_EUNSUPPORTED, "a storage type other than the volume's needs an FP32 volume");
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    const size_t vox = (size_t)G.nx * G.ny * G.nz;
    const size_t padded = fp_padded_elems(G.nx, G.ny, G.nz);
    const size_t need = padded * elem_size(storage);
    if (work_bytes < need || work == nullptr || !aligned16(work))
        return fail(PYRO_EWORKSPACE, "the staged forward projector needs a 16-byte aligned workspace of %zu bytes "
                                     "(got %zu)", need, work_bytes);
    if (batch == 0) return PYRO_OK;
    const int V = (int)G.beta.size();
    static thread_local FP3DParams p;
    bool column;
    if (int e = column_path(G, p, column)) return e;
    if (!column && storage != dt)
        return fail(PYRO_EUNSUPPORTED, "a separate storage type needs a circular-type trajectory (column kernels)");
    for (int b = 0; b < batch; ++b) {
        const char *vi = (const char *)vol + b * vox * elem_size(dt);
        if (column)
            PYRO_CUDA(launch_relayout_quad(vi, work, G.nx, G.ny, G.nz, dt, storage, as_stream(stream)));
        else
            PYRO_CUDA(launch_relayout_zmajor(vi, work, G.nx, G.ny, G.nz, dt, as_stream(stream)));
        for (int v0 = 0; v0 < V; v0 += kMaxViewsConeFP) {
            const int nvw = std::min(kMaxViewsConeFP, V - v0);
            if (int e = fill_fp3d(G, v0, nvw, p)) return e;
            if (column)
                PYRO_CUDA(launch_fp3d_column(work, sino, b, p, storage, dt, as_stream(stream)));
            else
                PYRO_CUDA(launch_fp3d_zmajor(work, sino, b, p, dt, as_stream(stream)));
        }
    }
    return PYRO_OK;
}

// the gathered adjoint serves a geometry whose every view has its camera's y
// axis along z (the rows of a detector column share their (x, y) point)
bool gather_path(const Geo3D &G)
{
    for (int v = 0; v < (int)G.beta.size(); ++v) {
        CamView c;
        GatherRows r;
        if (cam_view(G, v, c) != PYRO_OK || !c.col || gather_rows(G, c, r) != PYRO_OK || r.wrows == 0) return false;
    }
    return true;
}

// staged exact adjoint: per batch item the weighted sinogram is transposed
// into `work` ([view][k][l], so that a column's rows are contiguous), then
// the gather kernel writes the adjoint voxel by voxel (view chunks after the
// first add); geometries it does not serve take the per-sample scatter of
// fp3d (the workspace is then unused)
int fp3d_adjoint_staged(const void *sino, void *vol, int batch, const pyro_geom3d *g, void *work, size_t work_bytes,
                        pyro_dtype dt, void *stream)
{
    if (int e = check_io(sino, vol, batch, dt)) return e;
    if (dt != PYRO_F32) return fail(PYRO_EUNSUPPORTED, "the FP adjoint supports PYRO_F32 only");
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    const int V = (int)G.beta.size();
    const size_t vox = (size_t)G.nx * G.ny * G.nz, det = (size_t)G.nu * G.nv;
    const size_t need = (size_t)V * det * sizeof(float);
    if (work_bytes < need || work == nullptr || !aligned16(work))
        return fail(PYRO_EWORKSPACE, "the staged FP adjoint needs a 16-byte aligned workspace of %zu bytes (got %zu)",
                    need, work_bytes);
    if (batch == 0) return PYRO_OK;
    if (!gather_path(G)) return fp3d(sino, vol, batch, g, dt, true, stream);
    static thread_local FP3DParams p;
    static thread_local GatherParams gp;
    int *status = nullptr;
    PYRO_CUDA(status_word(&status));
    for (int b = 0; b < batch; ++b) {
        for (int v0 = 0; v0 < V; v0 += kMaxViewsConeFP) {
            if (int e = fill_fp3d(G, v0, std::min(kMaxViewsConeFP, V - v0), p)) return e;
            PYRO_CUDA(launch_weighted_transpose(sino, work, b, p, as_stream(stream)));
        }
        for (int v0 = 0; v0 < V; v0 += kMaxViewsGather) {
            if (int e = fill_gather(G, v0, std::min(kMaxViewsGather, V - v0), v0 > 0, gp)) return e;
            PYRO_CHECK(gather_smem_bytes(gp) <= 200 * 1024, "the gathered adjoint's tables exceed shared memory");
            PYRO_CUDA(launch_gather_adjoint(work, (float *)vol + b * vox, gp, status, as_stream(stream)));
        }
    }
    return PYRO_OK;
}

// Detector boxes of the TMA-staged BP: a bound, over every 32 x 8 x tz voxel
// tile and view of the chunk, on the extent of the tile's taps.  With the
// centred, SID-scaled map of fill_bp3d, u - cu = x / w and l - cv = y / w;
// along a segment inside the volume d(x/w) = (dx - (x/w) dw) / w, so the
// extent is at most (|dx| + max|x/w| |dw|) / min w, and likewise for l.  The
// extrema of x/w, y/w and w over the volume sit at its corners (linear-
// fractional maps with a positive depth).  False when the boxes do not fit.
bool tma_box_size(const BP3DParams &p, size_t elem, int tz, int &bu, int &bv)
{
    const double di = std::min(31, p.nx - 1), dj = std::min(7, p.ny - 1), dk = std::min(tz - 1, p.nz - 1);
    double ext_u = 0.0, ext_l = 0.0;
    for (int v = 0; v < p.n_views; ++v) {
        const float *P = p.P[v];
        double wmin = 1e300, xr = 0.0, yr = 0.0;
        for (int c = 0; c < 8; ++c) {
            const double i = (c & 1) ? p.nx - 1 : 0, j = (c & 2) ? p.ny - 1 : 0, k = (c & 4) ? p.nz - 1 : 0;
            const double x = P[0] * i + P[1] * j + P[2] * k + P[3];
            const double y = P[4] * i + P[5] * j + P[6] * k + P[7];
            const double w = P[8] * i + P[9] * j + P[10] * k + P[11];
            if (!(w > 0.0)) return false;
            wmin = std::min(wmin, w);
            xr = std::max(xr, std::fabs(x / w));
            yr = std::max(yr, std::fabs(y / w));
        }
        const double dw = std::fabs(P[8]) * di + std::fabs(P[9]) * dj;
        ext_u = std::max(ext_u, (std::fabs(P[0]) * di + std::fabs(P[1]) * dj + xr * dw) / wmin);
        ext_l = std::max(ext_l, (std::fabs(P[4]) * di + std::fabs(P[5]) * dj + std::fabs(P[6]) * dk + yr * dw) / wmin);
    }
    if (!(ext_u < 200.0 && ext_l < 200.0)) return false;
    // two taps, rounding margins and the 16-byte alignment of the box's x;
    // the box width is also the kernel's compile-time row pitch, 16 words
    // modulo the shared-memory banks: 80 or 144 floats, 96 or 160 halves
    const int align = (int)(16 / elem);
    const int need = ((int)std::ceil(ext_u) + 7 + align - 1) / align * align;
    const int p0 = elem == 4 ? 80 : 96, p1 = elem == 4 ? 144 : 160;
    bu = need <= p0 ? p0 : (need <= p1 ? p1 : 0);
    bv = (int)std::ceil(ext_l) + 4;
    return bu != 0 && bv <= 256;
}

// The TMA BP's tile depth and views per stage: four resident blocks (shared
// memory within a quarter of an SM's) first, then the deeper tile (half the
// per-view set-up per voxel), then two views per stage; if no plan fits four
// blocks, the one with the least shared memory.  Measured on the 256^3
// workload: 16-deep tiles with one view per stage 3.31 ms, 8-deep with two
// 4.37 ms, 8-deep with one 4.94 ms.  False when the TMA path does not apply
// (non-circular maps, a depth <= 0, boxes too large).
bool tma_plan(const BP3DParams &p, size_t elem, BPTmaPlan &pl)
{
    if (!p.z_invariant) return false;
    bool found = false;
    BPTmaPlan best{};
    size_t best_smem = 0;
    for (int tz : {16, 8}) {
        int bu = 0, bv = 0;
        if (!tma_box_size(p, elem, tz, bu, bv)) continue;
        for (int g : {2, 1}) {
            const size_t smem = bp3d_tma_smem_bytes(p.n_views, bu, bv, elem, g);
            if (smem <= 56 * 1024) {
                pl = {tz, bu, bv, g};
                return true;
            }
            if (!found || smem < best_smem) {
                best = {tz, bu, bv, g};
                best_smem = smem;
                found = true;
            }
        }
    }
    pl = best;
    return found && best_smem <= 200 * 1024;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (EncodeTiledFn)f;
    }();
    return fn;
}

// sinogram [views][nv][nu] (FP32, FP16 or BF16) as a 3D tensor map with
// bu x bv x 1 boxes; reads outside it return 0.  The row pitch must be a
// multiple of 16 bytes.
bool sino_tensor_map(const void *sino, pyro_dtype dt, int views, int nv, int nu, int bu, int bv, CUtensorMap &map)
{
    EncodeTiledFn fn = encode_tiled();
    const size_t es = elem_size(dt);
    if (!fn || ((uintptr_t)sino & 15) || ((size_t)nu * es) % 16) return false;
    const CUtensorMapDataType type = dt == PYRO_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                     : dt == PYRO_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)nu, (cuuint64_t)nv, (cuuint64_t)views};
    const cuuint64_t strides[2] = {(cuuint64_t)nu * es, (cuuint64_t)nu * nv * es};
    const cuuint32_t box[3] = {(cuuint32_t)bu, (cuuint32_t)bv, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(&map, type, 3, const_cast<void *>(sino), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int bp3d_impl(const void *sino, void *vol, int batch, const Geo3D &G, int wexp, float scale, pyro_dtype sino_dt,
              pyro_dtype vol_dt, void *stream)
{
    const int V = (int)G.beta.size();
    const size_t vox = (size_t)G.nx * G.ny * G.nz, det = (size_t)G.nu * G.nv;
    static thread_local BP3DParams p;
    const int zblocks = (G.nz + 7) / 8;  // the most z blocks of any BP kernel
    const int bstep = std::max(1, 65535 / zblocks);
    for (int v0 = 0; v0 < V; v0 += kMaxViewsConeBP) {
        const int nvw = std::min(kMaxViewsConeBP, V - v0);
        fill_bp3d(G, v0, nvw, wexp, scale, v0 > 0, p);
        BPTmaPlan plan{};
        const bool tma = (sino_dt == PYRO_F32 || sino_dt == vol_dt) && tma_plan(p, elem_size(sino_dt), plan);
        for (int b0 = 0; b0 < batch; b0 += bstep) {
            const int nb = std::min(bstep, batch - b0);
            const char *si = (const char *)sino + b0 * V * det * elem_size(sino_dt);
            char *vo = (char *)vol + b0 * vox * elem_size(vol_dt);
            CUtensorMap map;
            if (tma && sino_tensor_map(si, sino_dt, nb * V, G.nv, G.nu, plan.bu, plan.bv, map))
                PYRO_CUDA(launch_bp3d_tma(map, vo, nb, p, plan, sino_dt, vol_dt, as_stream(stream)));
            else
                PYRO_CUDA(launch_bp3d(si, vo, nb, p, sino_dt, vol_dt, as_stream(stream)));
        }
    }
    return PYRO_OK;
}

int bp3d(const void *sino, void *vol, int batch, const pyro_geom3d *g, pyro_bp_weight w, float scale, pyro_dtype dt,
         void *stream)
{
    if (int e = check_io(sino, vol, batch, dt)) return e;
    const int wexp = bp_weight_exp(w);
    PYRO_CHECK(wexp >= 0, "unknown back-projection weight %d", (int)w);
    PYRO_CHECK(std::isfinite(scale), "scale is not finite");
    if (wexp > 0) PYRO_CHECK(pos_finite(g ? g->sid : 0.0), "distance weights need SID > 0");
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    if (batch == 0) return PYRO_OK;
    return bp3d_impl(sino, vol, batch, G, wexp, scale, dt, dt, stream);
}

int bp3d_transpose(const void *vol, void *sino, int batch, const pyro_geom3d *g, pyro_bp_weight w, float scale,
                   pyro_dtype dt, void *stream)
{
    if (int e = check_io(vol, sino, batch, dt)) return e;
    if (dt != PYRO_F32) return fail(PYRO_EUNSUPPORTED, "the BP transpose supports PYRO_F32 only");
    const int wexp = bp_weight_exp(w);
    PYRO_CHECK(wexp >= 0, "unknown back-projection weight %d", (int)w);
    PYRO_CHECK(std::isfinite(scale), "scale is not finite");
    if (wexp > 0) PYRO_CHECK(pos_finite(g ? g->sid : 0.0), "distance weights need SID > 0");
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    if (batch == 0) return PYRO_OK;
    const int V = (int)G.beta.size();
    const size_t vox = (size_t)G.nx * G.ny * G.nz, det = (size_t)G.nu * G.nv;
    PYRO_CUDA(cudaMemsetAsync(sino, 0, sizeof(float) * batch * V * det, as_stream(stream)));
    static thread_local BP3DParams p;
    const int bstep = std::max(1, 65535 / G.nz);
    for (int v0 = 0; v0 < V; v0 += kMaxViewsConeBP) {
        const int nvw = std::min(kMaxViewsConeBP, V - v0);
        fill_bp3d(G, v0, nvw, wexp, scale, 0, p);
        for (int b0 = 0; b0 < batch; b0 += bstep) {
            const int nb = std::min(bstep, batch - b0);
            const float *vi = (const float *)vol + b0 * vox;
            float *so = (float *)sino + b0 * V * det;
            PYRO_CUDA(launch_bp3d_transpose(vi, so, nb, p, as_stream(stream)));
        }
    }
    return PYRO_OK;
}

}  // namespace

void set_last_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

int device_sm_count()
{
    static std::mutex mu;
    static std::map<int, int> counts;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    std::lock_guard<std::mutex> lock(mu);
    auto it = counts.find(dev);
    if (it != counts.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    counts[dev] = n;
    return n;
}

}  // namespace pyro

using namespace pyro;

extern "C" {

PYRO_API int pyro_fp_par2d(const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_dtype dtype,
                           void *stream)
{
    return fp2d(false, vol, sino, batch, g, dtype, stream);
}

PYRO_API int pyro_fp_fan2d(const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_dtype dtype,
                           void *stream)
{
    return fp2d(true, vol, sino, batch, g, dtype, stream);
}

PYRO_API int pyro_fp_cone3d(const void *vol, void *sino, int batch, const pyro_geom3d *g, pyro_dtype dtype,
                            void *stream)
{
    return fp3d(vol, sino, batch, g, dtype, false, stream);
}

PYRO_API int pyro_cone_projection_matrices(const pyro_geom3d *g, double *out)
{
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    PYRO_CHECK(out != nullptr, "out is NULL");
    std::copy(G.P.begin(), G.P.end(), out);
    return PYRO_OK;
}

PYRO_API size_t pyro_fp_cone3d_workspace_bytes(const pyro_geom3d *g, pyro_dtype dtype)
{
    if (!g || g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || !valid_dtype(dtype)) return 0;
    return fp_padded_elems(g->nx, g->ny, g->nz) * elem_size(dtype);
}

// ---- texture mode (the paper's fast mode, with its second copy) ----------
struct pyro_texture_s {
    int nx, ny, nz;  // array extent: (nx, ny, nz) of a volume, (nu, nv, n_views) of a layered sinogram
    bool layered;
    pyro_dtype dtype;
    cudaArray_t array;
    cudaTextureObject_t tex;
};

int texture_create(int nx, int ny, int nz, bool layered, pyro_dtype dtype, pyro_texture *out)
{
    PYRO_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    PYRO_CHECK(nx > 0 && ny > 0 && nz > 0, "texture extent must be positive (%d x %d x %d)", nx, ny, nz);
    if (dtype != PYRO_F32 && dtype != PYRO_F16)
        return fail(PYRO_EUNSUPPORTED, "textures hold PYRO_F32 or PYRO_F16 values");
    int dev = 0, w = 0, h = 0, d = 0;
    PYRO_CUDA(cudaGetDevice(&dev));
    if (layered) {
        PYRO_CUDA(cudaDeviceGetAttribute(&w, cudaDevAttrMaxTexture2DLayeredWidth, dev));
        PYRO_CUDA(cudaDeviceGetAttribute(&h, cudaDevAttrMaxTexture2DLayeredHeight, dev));
        PYRO_CUDA(cudaDeviceGetAttribute(&d, cudaDevAttrMaxTexture2DLayeredLayers, dev));
    } else {
        PYRO_CUDA(cudaDeviceGetAttribute(&w, cudaDevAttrMaxTexture3DWidth, dev));
        PYRO_CUDA(cudaDeviceGetAttribute(&h, cudaDevAttrMaxTexture3DHeight, dev));
        PYRO_CUDA(cudaDeviceGetAttribute(&d, cudaDevAttrMaxTexture3DDepth, dev));
    }
    PYRO_CHECK(nx <= w && ny <= h && nz <= d, "extent %d x %d x %d exceeds the device's %s texture limits %d x %d x %d",
               nx, ny, nz, layered ? "layered 2D" : "3D", w, h, d);
    const cudaChannelFormatDesc fd =
        cudaCreateChannelDesc(dtype == PYRO_F32 ? 32 : 16, 0, 0, 0, cudaChannelFormatKindFloat);
    auto *t = new pyro_texture_s{nx, ny, nz, layered, dtype, nullptr, 0};
    cudaError_t e = cudaMalloc3DArray(&t->array, &fd, make_cudaExtent(nx, ny, nz), layered ? cudaArrayLayered : 0);
    if (e != cudaSuccess) {
        delete t;
        return fail(PYRO_ECUDA, "cudaMalloc3DArray: %s", cudaGetErrorString(e));
    }
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof(rd));
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = t->array;
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof(td));  // border colour 0: the zero extension
    for (int a = 0; a < 3; ++a) td.addressMode[a] = cudaAddressModeBorder;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    e = cudaCreateTextureObject(&t->tex, &rd, &td, nullptr);
    if (e != cudaSuccess) {
        cudaFreeArray(t->array);
        delete t;
        return fail(PYRO_ECUDA, "cudaCreateTextureObject: %s", cudaGetErrorString(e));
    }
    *out = t;
    return PYRO_OK;
}

PYRO_API int pyro_texture_volume_create(int nx, int ny, int nz, pyro_dtype dtype, pyro_texture *out)
{
    return texture_create(nx, ny, nz, false, dtype, out);
}

PYRO_API int pyro_texture_sinogram_create(int nu, int nv, int n_views, pyro_dtype dtype, pyro_texture *out)
{
    return texture_create(nu, nv, n_views, true, dtype, out);
}

PYRO_API int pyro_texture_upload(pyro_texture t, const void *src, void *stream)
{
    PYRO_CHECK(t != nullptr && src != nullptr, "texture or source is NULL");
    const size_t es = elem_size(t->dtype);
    cudaMemcpy3DParms cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.srcPtr = make_cudaPitchedPtr(const_cast<void *>(src), (size_t)t->nx * es, (size_t)t->nx, (size_t)t->ny);
    cp.dstArray = t->array;
    cp.extent = make_cudaExtent((size_t)t->nx, (size_t)t->ny, (size_t)t->nz);
    cp.kind = cudaMemcpyDeviceToDevice;
    PYRO_CUDA(cudaMemcpy3DAsync(&cp, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_texture_destroy(pyro_texture t)
{
    if (t == nullptr) return PYRO_OK;
    const cudaError_t e1 = cudaDestroyTextureObject(t->tex);
    const cudaError_t e2 = cudaFreeArray(t->array);
    delete t;
    if (e1 != cudaSuccess || e2 != cudaSuccess)
        return fail(PYRO_ECUDA, "releasing a texture: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return PYRO_OK;
}

PYRO_API int pyro_fp_cone3d_tex(pyro_texture t, void *sino, const pyro_geom3d *g, pyro_dtype dtype, void *stream)
{
    PYRO_CHECK(t != nullptr && !t->layered, "not a volume texture");
    PYRO_CHECK(sino != nullptr && aligned16(sino), "sinogram pointer is NULL or not 16-byte aligned");
    PYRO_CHECK(valid_dtype(dtype), "unknown dtype %d", (int)dtype);
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    PYRO_CHECK(G.nx == t->nx && G.ny == t->ny && G.nz == t->nz,
               "geometry volume %d x %d x %d differs from the texture's %d x %d x %d", G.nx, G.ny, G.nz, t->nx, t->ny,
               t->nz);
    const int V = (int)G.beta.size();
    static thread_local FP3DParams p;
    for (int v0 = 0; v0 < V; v0 += kMaxViewsConeFP) {
        const int nvw = std::min(kMaxViewsConeFP, V - v0);
        if (int e = fill_fp3d(G, v0, nvw, p)) return e;
        PYRO_CUDA(launch_fp3d_tex(t->tex, sino, p, dtype, as_stream(stream)));
    }
    return PYRO_OK;
}

PYRO_API int pyro_bp_cone3d_tex(pyro_texture t, void *vol, const pyro_geom3d *g, pyro_bp_weight w, float scale,
                                pyro_dtype dtype, void *stream)
{
    PYRO_CHECK(t != nullptr && t->layered, "not a sinogram texture");
    PYRO_CHECK(vol != nullptr && aligned16(vol), "volume pointer is NULL or not 16-byte aligned");
    PYRO_CHECK(valid_dtype(dtype), "unknown dtype %d", (int)dtype);
    const int wexp = bp_weight_exp(w);
    PYRO_CHECK(wexp >= 0, "unknown back-projection weight %d", (int)w);
    PYRO_CHECK(std::isfinite(scale), "scale is not finite");
    if (wexp > 0) PYRO_CHECK(pos_finite(g ? g->sid : 0.0), "distance weights need SID > 0");
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    const int V = (int)G.beta.size();
    PYRO_CHECK(G.nu == t->nx && G.nv == t->ny && V == t->nz,
               "geometry sinogram %d views x %d x %d differs from the texture's %d x %d x %d", V, G.nv, G.nu, t->nz,
               t->ny, t->nx);
    static thread_local BP3DParams p;
    for (int v0 = 0; v0 < V; v0 += kMaxViewsConeBP) {
        fill_bp3d(G, v0, std::min(kMaxViewsConeBP, V - v0), wexp, scale, v0 > 0, p);
        PYRO_CUDA(launch_bp3d_tex(t->tex, vol, p, dtype, as_stream(stream)));
    }
    return PYRO_OK;
}

PYRO_API int pyro_fp_cone3d_ws(const void *vol, void *sino, int batch, const pyro_geom3d *g, void *workspace,
                               size_t workspace_bytes, pyro_dtype dtype, void *stream)
{
    return fp3d_staged(vol, sino, batch, g, workspace, workspace_bytes, dtype, dtype, stream);
}

PYRO_API int pyro_fp_cone3d_ws_storage(const void *vol, void *sino, int batch, const pyro_geom3d *g, void *workspace,
                                       size_t workspace_bytes, pyro_dtype dtype, pyro_dtype storage, void *stream)
{
    return fp3d_staged(vol, sino, batch, g, workspace, workspace_bytes, dtype, storage, stream);
}

PYRO_API size_t pyro_fp2d_workspace_bytes(const pyro_geom2d *g, int batch, pyro_dtype dtype)
{
    if (!g || g->nx <= 0 || g->ny <= 0 || batch < 0 || !valid_dtype(dtype)) return 0;
    return (size_t)g->nx * g->ny * elem_size(dtype) * (size_t)std::max(batch, 1);
}

PYRO_API int pyro_fp_par2d_ws(const void *vol, void *sino, int batch, const pyro_geom2d *g, void *workspace,
                              size_t workspace_bytes, pyro_dtype dtype, void *stream)
{
    PYRO_CHECK(workspace != nullptr, "workspace is NULL");
    return fp2d(false, vol, sino, batch, g, dtype, stream, workspace, workspace_bytes);
}

PYRO_API int pyro_fp_fan2d_ws(const void *vol, void *sino, int batch, const pyro_geom2d *g, void *workspace,
                              size_t workspace_bytes, pyro_dtype dtype, void *stream)
{
    PYRO_CHECK(workspace != nullptr, "workspace is NULL");
    return fp2d(true, vol, sino, batch, g, dtype, stream, workspace, workspace_bytes);
}

PYRO_API int pyro_fpT_par2d_ws(const void *sino, void *vol, int batch, const pyro_geom2d *g, void *workspace,
                               size_t workspace_bytes, pyro_dtype dtype, void *stream)
{
    PYRO_CHECK(workspace != nullptr, "workspace is NULL");
    return fp2d_adjoint(false, sino, vol, batch, g, dtype, stream, workspace, workspace_bytes);
}

PYRO_API int pyro_fpT_fan2d_ws(const void *sino, void *vol, int batch, const pyro_geom2d *g, void *workspace,
                               size_t workspace_bytes, pyro_dtype dtype, void *stream)
{
    PYRO_CHECK(workspace != nullptr, "workspace is NULL");
    return fp2d_adjoint(true, sino, vol, batch, g, dtype, stream, workspace, workspace_bytes);
}

PYRO_API int pyro_fpT_par2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_dtype dtype,
                            void *stream)
{
    return fp2d_adjoint(false, sino, vol, batch, g, dtype, stream);
}

PYRO_API int pyro_fpT_fan2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_dtype dtype,
                            void *stream)
{
    return fp2d_adjoint(true, sino, vol, batch, g, dtype, stream);
}

PYRO_API int pyro_fpT_cone3d(const void *sino, void *vol, int batch, const pyro_geom3d *g, pyro_dtype dtype,
                             void *stream)
{
    return fp3d(sino, vol, batch, g, dtype, true, stream);
}

PYRO_API size_t pyro_fpT_cone3d_workspace_bytes(const pyro_geom3d *g)
{
    if (!g || g->nu <= 0 || g->nv <= 0 || g->n_views <= 0) return 0;
    return (size_t)g->n_views * g->nu * g->nv * sizeof(float);
}

PYRO_API int pyro_fpT_cone3d_ws(const void *sino, void *vol, int batch, const pyro_geom3d *g, void *workspace,
                                size_t workspace_bytes, pyro_dtype dtype, void *stream)
{
    return fp3d_adjoint_staged(sino, vol, batch, g, workspace, workspace_bytes, dtype, stream);
}

PYRO_API int pyro_bp_par2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_bp_weight w,
                           float scale, pyro_dtype dtype, void *stream)
{
    return bp2d(false, sino, vol, batch, g, w, scale, dtype, dtype, stream);
}

PYRO_API int pyro_bp_fan2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_bp_weight w,
                           float scale, pyro_dtype dtype, void *stream)
{
    return bp2d(true, sino, vol, batch, g, w, scale, dtype, dtype, stream);
}

PYRO_API int pyro_bp_cone3d(const void *sino, void *vol, int batch, const pyro_geom3d *g, pyro_bp_weight w,
                            float scale, pyro_dtype dtype, void *stream)
{
    return bp3d(sino, vol, batch, g, w, scale, dtype, stream);
}

PYRO_API int pyro_bpT_par2d(const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_bp_weight w,
                            float scale, pyro_dtype dtype, void *stream)
{
    return bp2d_transpose(false, vol, sino, batch, g, w, scale, dtype, stream);
}

PYRO_API int pyro_bpT_fan2d(const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_bp_weight w,
                            float scale, pyro_dtype dtype, void *stream)
{
    return bp2d_transpose(true, vol, sino, batch, g, w, scale, dtype, stream);
}

PYRO_API int pyro_bpT_cone3d(const void *vol, void *sino, int batch, const pyro_geom3d *g, pyro_bp_weight w,
                             float scale, pyro_dtype dtype, void *stream)
{
    return bp3d_transpose(vol, sino, batch, g, w, scale, dtype, stream);
}

PYRO_API int pyro_weights2d(void *sino, int batch, const pyro_geom2d *g, int cosine, pyro_redund redund,
                            pyro_dtype dtype, void *stream)
{
    if (int e = check_io(sino, sino, batch, dtype)) return e;
    Geo2D G;
    if (int e = prep2d(g, false, G)) return e;
    WeightParams w;
    static thread_local BetaTable bt;
    if (int e = fill_weights(G.nu, 1, G.su, 0.0, g->sdd, G.beta, G.range, cosine, redund, w, bt)) return e;
    if (batch == 0) return PYRO_OK;
    PYRO_CUDA(launch_weights(sino, batch, w, bt, dtype, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_weights3d(void *sino, int batch, const pyro_geom3d *g, int cosine, pyro_redund redund,
                            pyro_dtype dtype, void *stream)
{
    if (int e = check_io(sino, sino, batch, dtype)) return e;
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    WeightParams w;
    static thread_local BetaTable bt;
    if (int e = fill_weights(G.nu, G.nv, G.su, G.sv, G.sdd, G.beta, G.range, cosine, redund, w, bt)) return e;
    if (batch == 0) return PYRO_OK;
    PYRO_CUDA(launch_weights(sino, batch, w, bt, dtype, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_weights3d_table(void *sino, int batch, const pyro_geom3d *g, const float *table, int cosine,
                                  pyro_dtype dtype, void *stream)
{
    if (int e = check_io(sino, sino, batch, dtype)) return e;
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    if (batch > 0) PYRO_CHECK(table != nullptr, "table is NULL");
    WeightParams w;
    static thread_local BetaTable bt;
    if (int e = fill_weights(G.nu, G.nv, G.su, G.sv, G.sdd, G.beta, G.range, cosine, PYRO_REDUND_NONE, w, bt)) return e;
    if (batch == 0) return PYRO_OK;
    PYRO_CUDA(launch_weights_table(sino, batch, w, table, dtype, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_redundancy_grad(const float *a, const float *g, float *out, int batch, int n_views, int nv, int nu,
                                  void *stream)
{
    PYRO_CHECK(batch >= 0 && n_views > 0 && nv > 0 && nu > 0, "sizes must be positive (batch >= 0)");
    PYRO_CHECK(n_views <= 65535, "n_views=%d above 65535", n_views);
    PYRO_CHECK(out != nullptr, "out is NULL");
    if (batch > 0) PYRO_CHECK(a != nullptr && g != nullptr, "input pointer is NULL");
    if (batch == 0) {
        PYRO_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)n_views * nu, as_stream(stream)));
        return PYRO_OK;
    }
    PYRO_CUDA(launch_redundancy_grad(a, g, out, batch, n_views, nv, nu, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_filter_pad_length(int nu)
{
    return nu > 0 ? pad_length(nu) : 0;
}

PYRO_API int pyro_filter_spectrum(pyro_filter kind, int nu, double tau, float *K_out)
{
    PYRO_CHECK(K_out != nullptr, "K_out is NULL");
    PYRO_CHECK(nu > 0 && nu <= kMaxPadLength / 2, "nu=%d outside [1, %d]", nu, kMaxPadLength / 2);
    PYRO_CHECK(kind == PYRO_RAMLAK || kind == PYRO_RAMP || kind == PYRO_SHEPP_LOGAN, "not a built-in filter: %d",
               (int)kind);
    PYRO_CHECK(pos_finite(tau), "tau must be positive and finite");
    const std::vector<float> &K = builtin_K(kind, pad_length(nu), tau);
    std::copy(K.begin(), K.end(), K_out);
    return PYRO_OK;
}

PYRO_API int pyro_filter_rows(const void *in, void *out, long n_rows, int nu, double tau, pyro_filter kind,
                              const float *custom_K, pyro_dtype dtype, void *stream)
{
    if (int e = check_io(in, out, n_rows, dtype)) return e;
    static thread_local FilterParams p;
    if (int e = fill_filter(n_rows, nu, tau, kind, custom_K, p)) return e;
    if (n_rows == 0) return PYRO_OK;
    PYRO_CUDA(launch_filter(in, out, p, nullptr, kind == PYRO_FILTER_CUSTOM ? custom_K : nullptr, dtype, dtype,
                            as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_filter_grad_K(const float *p, const float *g, float *dK, long n_rows, int nu, void *stream)
{
    if (int e = check_io(p, g, n_rows, PYRO_F32)) return e;
    PYRO_CHECK(dK != nullptr, "dK is NULL");
    PYRO_CHECK(n_rows >= 0 && nu > 0 && nu <= kMaxPadLength / 2, "bad row shape");
    const int pn = pad_length(nu);
    if (n_rows == 0) {
        PYRO_CUDA(cudaMemsetAsync(dK, 0, sizeof(float) * (pn / 2 + 1), as_stream(stream)));
        return PYRO_OK;
    }
    PYRO_CUDA(launch_filter_grad_K(p, g, dK, n_rows, nu, pn, log2_exact(pn), as_stream(stream)));
    return PYRO_OK;
}

PYRO_API size_t pyro_fdk_workspace_bytes(const pyro_geom3d *g, int batch)
{
    if (!g || batch < 0) return 0;
    return sizeof(float) * (size_t)batch * (size_t)std::max(g->n_views, 0) * (size_t)std::max(g->nv, 0) *
           (size_t)std::max(g->nu, 0);
}

PYRO_API int pyro_fdk(const void *sino, void *vol, int batch, const pyro_geom3d *g, pyro_filter kind,
                      const float *custom_K, pyro_redund redund, void *workspace, size_t workspace_bytes,
                      pyro_dtype dtype, void *stream)
{
    if (int e = check_io(sino, vol, batch, dtype)) return e;
    Geo3D G;
    if (int e = prep3d(g, G)) return e;
    PYRO_CHECK(pos_finite(G.sid) && pos_finite(G.sdd) && G.sdd > G.sid, "FDK needs 0 < SID < SDD");
    PYRO_CHECK(std::isfinite(G.range) && G.range != 0.0, "FDK needs the angular range (scale range / n_views)");
    const size_t need = pyro_fdk_workspace_bytes(g, batch);
    if (workspace_bytes < need || (need > 0 && (workspace == nullptr || !aligned16(workspace))))
        return fail(PYRO_EWORKSPACE, "FDK needs a 16-byte aligned workspace of %zu bytes (got %zu)", need,
                    workspace_bytes);
    const int V = (int)G.beta.size();
    static thread_local FilterParams p;
    static thread_local BetaTable bt;
    if (int e = fill_filter((long)batch * V * G.nv, G.nu, G.su * G.sid / G.sdd, kind, custom_K, p)) return e;
    if (int e = fill_weights(G.nu, G.nv, G.su, G.sv, G.sdd, G.beta, G.range, 1, redund, p.w, bt)) return e;
    p.apply_weights = 1;
    p.rows_per_view = G.nv;
    p.n_views = V;
    if (batch == 0) return PYRO_OK;
    PYRO_CUDA(launch_filter(sino, workspace, p, &bt, kind == PYRO_FILTER_CUSTOM ? custom_K : nullptr, dtype, PYRO_F32,
                            as_stream(stream)));
    return bp3d_impl(workspace, vol, batch, G, 2, (float)(std::fabs(G.range) / V), PYRO_F32, dtype, stream);
}

PYRO_API size_t pyro_fbp2d_workspace_bytes(const pyro_geom2d *g, int batch)
{
    if (!g || batch < 0) return 0;
    return sizeof(float) * (size_t)batch * (size_t)std::max(g->n_views, 0) * (size_t)std::max(g->nu, 0);
}

static int fbp2d(bool fan, const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_filter kind,
                 const float *custom_K, pyro_redund redund, void *workspace, size_t workspace_bytes, pyro_dtype dtype,
                 void *stream)
{
    if (int e = check_io(sino, vol, batch, dtype)) return e;
    Geo2D G;
    if (int e = prep2d(g, fan, G)) return e;
    const size_t need = pyro_fbp2d_workspace_bytes(g, batch);
    if (workspace_bytes < need || (need > 0 && (workspace == nullptr || !aligned16(workspace))))
        return fail(PYRO_EWORKSPACE, "FBP needs a 16-byte aligned workspace of %zu bytes (got %zu)", need,
                    workspace_bytes);
    const int V = (int)G.beta.size();
    static thread_local FilterParams p;
    static thread_local BetaTable bt;
    const double tau = fan ? G.su * G.sid / G.sdd : G.su;
    if (int e = fill_filter((long)batch * V, G.nu, tau, kind, custom_K, p)) return e;
    if (fan) {
        PYRO_CHECK(std::isfinite(G.range) && G.range != 0.0, "fan FBP needs the angular range");
        if (int e = fill_weights(G.nu, 1, G.su, 0.0, G.sdd, G.beta, G.range, 1, redund, p.w, bt)) return e;
        p.apply_weights = 1;
        p.rows_per_view = 1;
        p.n_views = V;
    }
    if (batch == 0) return PYRO_OK;
    PYRO_CUDA(launch_filter(sino, workspace, p, fan ? &bt : nullptr, kind == PYRO_FILTER_CUSTOM ? custom_K : nullptr,
                            dtype, PYRO_F32, as_stream(stream)));
    const double pi = 3.14159265358979323846;
    const float scale = (float)(fan ? std::fabs(G.range) / V : pi / V);
    static thread_local BP2DParams bp;
    for (int v0 = 0; v0 < V; v0 += kMaxViewsBP2D) {
        const int nvw = std::min(kMaxViewsBP2D, V - v0);
        fill_bp2d(G, v0, nvw, fan ? 2 : 0, scale, bp);
        for (int b0 = 0; b0 < batch; b0 += 65535) {
            const int nb = std::min(65535, batch - b0);
            const float *si = (const float *)workspace + (size_t)b0 * V * G.nu;
            char *vo = (char *)vol + (size_t)b0 * G.nx * G.ny * elem_size(dtype);
            PYRO_CUDA(launch_bp2d(si, vo, nb, bp, PYRO_F32, dtype, v0 > 0, as_stream(stream)));
        }
    }
    return PYRO_OK;
}

PYRO_API int pyro_fbp_par2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_filter kind,
                            const float *custom_K, void *workspace, size_t workspace_bytes, pyro_dtype dtype,
                            void *stream)
{
    return fbp2d(false, sino, vol, batch, g, kind, custom_K, PYRO_REDUND_NONE, workspace, workspace_bytes, dtype,
                 stream);
}

PYRO_API int pyro_fbp_fan2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_filter kind,
                            const float *custom_K, pyro_redund redund, void *workspace, size_t workspace_bytes,
                            pyro_dtype dtype, void *stream)
{
    return fbp2d(true, sino, vol, batch, g, kind, custom_K, redund, workspace, workspace_bytes, dtype, stream);
}

PYRO_API int pyro_tv(const float *x, float *grad, const float *base, float alpha, float lambda, float *value,
                     int batch, int nz, int ny, int nx, float eps, void *stream)
{
    PYRO_CHECK(batch >= 0 && nz > 0 && ny > 0 && nx > 0, "bad volume shape");
    PYRO_CHECK(batch <= 65535, "batch must be <= 65535");
    PYRO_CHECK(std::isfinite(eps) && eps > 0.0f, "eps must be positive");
    PYRO_CHECK(std::isfinite(alpha) && std::isfinite(lambda), "alpha / lambda must be finite");
    if (batch == 0) return PYRO_OK;
    PYRO_CHECK(x != nullptr && (grad != nullptr || value != nullptr), "need x and at least one of grad / value");
    PYRO_CHECK(aligned16(x) && aligned16(grad) && aligned16(base), "device pointers must be 16-byte aligned");
    PYRO_CUDA(launch_tv(x, grad, base, alpha, lambda, value, batch, nz, ny, nx, eps, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_axpby(const float *x, float *y, long n, float a, float b, void *stream)
{
    PYRO_CHECK(n >= 0, "n must be >= 0");
    if (n == 0) return PYRO_OK;
    PYRO_CHECK(x != nullptr && y != nullptr, "NULL pointer");
    PYRO_CUDA(launch_axpby(x, y, n, a, b, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_dot(const float *a, const float *b, long n, float *out, void *stream)
{
    PYRO_CHECK(n >= 0 && out != nullptr, "bad arguments");
    if (n > 0) PYRO_CHECK(a != nullptr && b != nullptr, "NULL pointer");
    if (n == 0) {
        PYRO_CUDA(cudaMemsetAsync(out, 0, sizeof(float), as_stream(stream)));
        return PYRO_OK;
    }
    PYRO_CUDA(launch_dot(a, b, n, out, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_bb_dots(const float *x, const float *x_prev, const float *g, const float *g_prev, long n,
                          float *dots, void *stream)
{
    PYRO_CHECK(n >= 0 && dots != nullptr, "bad arguments");
    if (n > 0) PYRO_CHECK(x && x_prev && g && g_prev, "NULL pointer");
    if (n == 0) {
        PYRO_CUDA(cudaMemsetAsync(dots, 0, 2 * sizeof(float), as_stream(stream)));
        return PYRO_OK;
    }
    PYRO_CUDA(launch_bb_dots(x, x_prev, g, g_prev, n, dots, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_bb_update(float *x, float *x_prev, const float *g, float *g_prev, long n, const float *dots,
                            float alpha0, float alpha_max, int first, float *alpha_out, void *stream)
{
    PYRO_CHECK(n >= 0, "n must be >= 0");
    PYRO_CHECK(std::isfinite(alpha0) && std::isfinite(alpha_max) && alpha0 >= 0 && alpha_max >= 0,
               "step bounds must be finite and >= 0");
    if (!first) PYRO_CHECK(dots != nullptr, "dots is NULL");
    if (n > 0) PYRO_CHECK(x && x_prev && g && g_prev, "NULL pointer");
    if (n == 0) return PYRO_OK;
    PYRO_CUDA(launch_bb_update(x, x_prev, g, g_prev, n, dots, alpha0, alpha_max, first, alpha_out,
                               as_stream(stream)));
    return PYRO_OK;
}

static int conv_dims_ok(int batch, int nz, int ny, int nx, int cin, int cout)
{
    PYRO_CHECK(batch >= 0 && nz > 0 && ny > 0 && nx > 0, "bad activation shape");
    PYRO_CHECK(conv_supported(cin, cout), "unsupported channel pair (%d, %d)", cin, cout);
    if (cin == 16 && nx % 128 == 0) {
        // rows of 128 output voxels along x: any nz, ny
        PYRO_CHECK((long)batch * nz * ny * (nx / 128) < (1L << 31), "too many voxel rows");
    } else {
        // blocks of 128 output voxels: TX = min(nx, 64), TY = min(ny, 128 / TX), TZ = 128 / (TX TY)
        PYRO_CHECK(nx == 8 || nx == 16 || nx == 32 || (nx >= 64 && nx % 64 == 0),
                   "nx=%d must be 8, 16, 32 or a multiple of 64", nx);
        const int tx = nx >= 64 ? 64 : nx;
        const int ty = std::min(ny, 128 / tx);
        PYRO_CHECK(ny % ty == 0 && (128 / tx) % ty == 0, "ny=%d does not tile by %d", ny, ty);
        const int tz = 128 / (tx * ty);
        PYRO_CHECK(nz % tz == 0, "nz=%d must be a multiple of %d", nz, tz);
        PYRO_CHECK((long)batch * (nz / tz) * (ny / ty) * (nx / tx) < (1L << 31), "too many voxel tiles");
    }
    return PYRO_OK;
}

PYRO_API int pyro_conv3d(const void *x, const void *w, const float *bias, void *y, int batch, int nz, int ny, int nx,
                         int cin, int cout, int relu, void *stream)
{
    if (int e = conv_dims_ok(batch, nz, ny, nx, cin, cout)) return e;
    if (batch == 0) return PYRO_OK;
    PYRO_CHECK(x && w && y, "NULL pointer");
    PYRO_CHECK(aligned16(x) && aligned16(w) && aligned16(y) && aligned16(bias), "pointers must be 16-byte aligned");
    PYRO_CUDA(launch_conv3d(x, w, bias, y, batch, nz, ny, nx, cin, cout, relu, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_conv3d_wgrad(const void *x, const void *dy, float *dw, int batch, int nz, int ny, int nx, int cin,
                               int cout, void *stream)
{
    if (int e = conv_dims_ok(batch, nz, ny, nx, cin, cout)) return e;
    PYRO_CHECK(dw != nullptr, "NULL pointer");
    if (batch == 0) {
        PYRO_CUDA(cudaMemsetAsync(dw, 0, sizeof(float) * 27 * cin * cout, as_stream(stream)));
        return PYRO_OK;
    }
    PYRO_CHECK(x && dy, "NULL pointer");
    PYRO_CHECK(aligned16(x) && aligned16(dy), "pointers must be 16-byte aligned");
    PYRO_CUDA(launch_conv3d_wgrad(x, dy, dw, batch, nz, ny, nx, cin, cout, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_conv3d_flip_weights(const void *w, void *wf, int cin, int cout, void *stream)
{
    PYRO_CHECK(w && wf && cin > 0 && cout > 0, "bad arguments");
    PYRO_CUDA(launch_weight_flip(w, wf, cin, cout, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_cnn_op(int op, const void *a, const void *b, void *y, const float *f, long n, int nz, int ny, int nx,
                         int c, void *stream)
{
    PYRO_CHECK(op >= 0 && op <= 8, "unknown CNN op %d", op);
    PYRO_CHECK(n >= 0, "n must be >= 0");
    if (n == 0) return PYRO_OK;
    PYRO_CHECK(a && y, "NULL pointer");
    if (op == PYRO_CNN_ADD) PYRO_CHECK(b != nullptr, "ADD needs b");
    if (op == PYRO_CNN_RESIDUAL) PYRO_CHECK(f != nullptr, "RESIDUAL needs f");
    if (op >= 1 && op <= 4) {
        PYRO_CHECK(nz > 0 && ny > 0 && nx > 0 && c > 0, "bad shape");
        if (op <= 2) PYRO_CHECK(nz % 2 == 0 && ny % 2 == 0 && nx % 2 == 0, "pooling needs even dims");
    }
    PYRO_CUDA(launch_cnn_elementwise(op, a, b, y, f, n, nz, ny, nx, c, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_cnn_bias_grad(const void *dy, float *db, long nvox, int c, void *stream)
{
    PYRO_CHECK(dy && db && nvox >= 0 && c > 0 && c <= 65535, "bad arguments");
    PYRO_CUDA(launch_bias_grad(dy, db, nvox, c, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_cnn_mse(const float *out, const float *target, void *grad, float *loss, long n, void *stream)
{
    PYRO_CHECK(out && target && loss && n > 0, "bad arguments");
    PYRO_CUDA(launch_mse(out, target, grad, loss, n, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_cnn_adam(float *p, const float *g, float *m, float *v, void *p16, long n, float lr, float beta1,
                           float beta2, float eps, int step, void *stream)
{
    PYRO_CHECK(p && g && m && v && n >= 0 && step >= 1, "bad arguments");
    PYRO_CHECK(std::isfinite(lr) && beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps > 0, "bad Adam settings");
    if (n == 0) return PYRO_OK;
    PYRO_CUDA(launch_adam(p, g, m, v, p16, n, lr, beta1, beta2, eps, step, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_sync_status(void *stream)
{
    PYRO_CUDA(cudaStreamSynchronize(as_stream(stream)));
    PYRO_CUDA(cudaGetLastError());
    // the word a bounded device-side wait sets when it gives up (TMA-staged BP)
    int *word = nullptr;
    PYRO_CUDA(status_word(&word));
    int flag = 0;
    PYRO_CUDA(cudaMemcpy(&flag, word, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        PYRO_CUDA(cudaMemset(word, 0, sizeof(int)));
        if (flag & 1) return fail(PYRO_ETIMEOUT, "a device-side wait gave up; the results of that call are not valid");
        return fail(PYRO_ECUDA, "a kernel's shared table outgrew its host-computed bound; the results of that call "
                                "are not valid");
    }
    return PYRO_OK;
}

PYRO_API int pyro_probe_gather(const void *buf, size_t bytes, int loads_per_thread, long threads, unsigned *sink,
                               void *stream)
{
    PYRO_CHECK(buf != nullptr && sink != nullptr, "NULL pointer");
    PYRO_CHECK(aligned16(buf) && bytes >= 16 && bytes / 16 <= 0xFFFFFFFFull, "buffer must be 16-byte aligned, 16 B .. 64 GiB");
    PYRO_CHECK(loads_per_thread > 0 && threads > 0 && threads <= (1L << 31), "bad probe size");
    PYRO_CUDA(launch_gather_probe(buf, (unsigned)(bytes / 16), loads_per_thread, sink, threads, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API int pyro_selftest_wait_timeout(int limit_ms, void *stream)
{
    PYRO_CHECK(limit_ms >= 1 && limit_ms <= 1000, "limit_ms=%d outside [1, 1000]", limit_ms);
    PYRO_CUDA(launch_wait_timeout_probe((unsigned long long)limit_ms * 1000000ull, as_stream(stream)));
    return PYRO_OK;
}

PYRO_API const char *pyro_last_error(void)
{
    return g_last_error.c_str();
}

PYRO_API const char *pyro_version(void)
{
    return "pyro-gb300 0.1 (sm_103a)";
}

}  // extern "C"
