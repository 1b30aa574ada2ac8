// Internal declarations shared by the host API (pyro_api.cpp) and the CUDA
// kernels.  Per-view geometry travels to the kernels as __grid_constant__
// kernel parameters (read through the constant cache, warp-uniform in every
// kernel), so concurrent calls on different streams never share state and
// the library needs no device allocation of its own.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "pyro.h"

namespace pyro {

// Kernel-parameter space is 32764 bytes; these caps keep every parameter
// pack below it.  Longer trajectories are processed in chunks of views.
constexpr int kMaxViews2D = 1024;    // 2D weights: views of one beta table
constexpr int kMaxViewsBP2D = 512;   // 2D BP: 12 floats per view (map as hi/lo pairs)
constexpr int kMaxViewsConeBP = 300; // cone BP: 24 floats per view (map as hi/lo pairs)
constexpr int kMaxViewsConeFP = 200; // cone FP: 34 floats per view (hi/lo pairs)
constexpr int kMaxPadLength = 8192;  // filter: pn <= 8192, so nu <= 4096

// ---------------------------------------------------------------- FP 2D --
// Ray of bin k in view j: sample m at p(k) + m q(k) in pixel-index units,
// with p and q affine in k; parallel beam a = u e_u, g = c; fan beam
// a = (SID u / SDD) e_u (the sample on the iso-centre's depth plane),
// g = c + (u / SDD) e_u.  The host evaluates the affine coefficients in FP64
// and passes them as FP32 pairs (hi + lo); the kernels anchor the sample
// positions every kFPSegment samples in float-float (see FP3DParams).
constexpr int kMaxViewsFP2D = 384;   // 2D FP: 18 floats per view
struct FP2DLine {
    float p0x, pkx, p0y, pky;  // p(k) = p0 + k pk
    float q0x, qkx, q0y, qky;  // q(k) = q0 + k qk
};

struct FP2DParams {
    int nx, ny, nu, n_views;   // n_views in this chunk
    int view0;                 // first view of this chunk (sinogram offset)
    int views_total;           // views in the full sinogram
    int fan;
    int M;                     // samples m = -M..M around the closest approach
    float su, cu;              // bin spacing, (nu-1)/2
    float sdd;
    float dt;
    float2 dir[kMaxViewsFP2D];    // central-ray vector c_j = (cos b_j, sin b_j)
    FP2DLine ln[kMaxViewsFP2D];   // the rays' affine maps, FP32
    FP2DLine lnlo[kMaxViewsFP2D]; // FP64 maps - ln
};

// ---------------------------------------------------------------- FP 3D --
// Cone ray of pixel (k, l) in camera coordinates q = K^-1 (k, l, 1) (P = K R
// [I | -S] after an RQ split done in FP64 on the host); the closest approach
// of the ray to the iso-centre is
//   B_cam = s_perp - (s_perp.q) q/|q|^2 + s3 (-q_x, -q_y, q_x^2+q_y^2)/|q|^2
// with S_cam = R S = (s_perp, s3), free of cancellation.  W = diag(1/s) R^T
// takes camera vectors to voxel-index units.
struct ConeFPView {
    float W[9];                // row-major 3x3
    float a0, a1, a2;          // q_x = a0 k + a1 l + a2
    float b0, b2;              // q_y = b0 l + b2
    float s1, s2, s3;          // source in camera coordinates
};

// The FP64 set-up travels as FP32 pairs (v + vlo, dt + dt_lo): the kernels
// evaluate each ray's sample positions in float-float arithmetic every
// kFPSegment depth planes (an integer cell plus an FP32 fraction per axis) and
// step in FP32 from there, so a sample position near voxel index 500 keeps
// ~1e-6 voxel where an absolute FP32 index carries ~3e-5.
constexpr int kFPSegment = 64;
// The column kernels' padded z-major quad copy of the volume: cells
// [ny + 2 P][nx + 2 P][nz + 2], P = kFPPadXY zero voxels before and after the
// data in x and y and one in z; cell (x, y, z) holds the four voxels (x, y),
// (x + 1, y), (x, y + 1), (x + 1, y + 1) at z (one load per plane).  Two in x
// and y keep the taps inside the copy when an anchored sample lands one cell
// beyond the FP32 range test that chose it.
constexpr int kFPPadXY = 2;
inline size_t fp_padded_cells(int nx, int ny, int nz)
{
    return (size_t)(nx + 2 * kFPPadXY) * (ny + 2 * kFPPadXY) * (nz + 2);
}
inline size_t fp_padded_elems(int nx, int ny, int nz)  // elements of the quad copy
{
    return 4 * fp_padded_cells(nx, ny, nz);
}
struct FP3DParams {
    int nx, ny, nz, nu, nv, n_views, view0, views_total;
    int column_shared;         // every view: rows of a detector column share (x, y) (see fill_fp3d)
    int pair_rows;             // > 0: rows per window of the two-rays-per-lane column kernels (33..64)
    int M;
    float cx, cy, cz;          // (n-1)/2 per axis
    float dt, dt_lo;
    ConeFPView v[kMaxViewsConeFP];
    ConeFPView vlo[kMaxViewsConeFP];  // FP64 set-up - v
};

// --------------------------------------------------- gathered cone adjoint --
// Per view, for circular-type trajectories (the detector's v axis along z),
// in voxel-index units: the (x, y) point of column k on depth plane m,
// X = px0 + k pxk + m (qx0 + k qxk) (and Y alike), the z of row l there,
// z = A + m C + (B + m D) l, the detector column coordinate of the voxel
// column (x, y), (u0 + ui x + uj y) / (w0 + wi x + wj y), and its depth-plane
// coordinate mc + mi x + mj y.  Pairs are FP64 values as FP32 hi/lo.
constexpr int kGatherWarps = 4;   // warps per block (32 z voxels each)
// voxel columns per tile side: 6 (fewer border points per column), or 4 when
// 6-column tiles would give the launch fewer than 1024 blocks (small volumes:
// 128^3 has 484 such blocks for 152 SMs)
inline int gather_tile(int nx, int ny, int nz)
{
    const long blocks6 = (long)((nx + 5) / 6) * ((ny + 5) / 6) * ((nz + 32 * kGatherWarps - 1) / (32 * kGatherWarps));
    return blocks6 >= 1024 ? 6 : 4;
}
constexpr int kMaxViewsGather = 200;
struct GatherView {
    float px0[2], pxk[2], py0[2], pyk[2];
    float qx0[2], qxk[2], qy0[2], qyk[2];
    float A[2], B[2], C[2], D[2];
    float u0, ui, uj, w0, wi, wj;
    float mc, mi, mj, pad;
};

struct GatherParams {
    int nx, ny, nz, nu, nv, n_views, view0, views_total, M;
    int accumulate;                  // add into the output (view chunks after the first)
    int kmax, plmax;                 // columns and depth planes that can reach a tile (host bounds)
    int wrows;                       // rows of a lane's window (a multiple of 4, at most 32)
    int sc;                          // staged floats per warp (a column's rows at least)
    int tile;                        // voxel columns per tile side (gather_tile)
    GatherView v[kMaxViewsGather];
};

// ------------------------------------------------------------- BP 2D/3D --
// Voxel-index to detector map, pre-scaled on the host: for voxel (i, j[, z])
//   x = r0 . (i, j[, z], 1),  w = r2 . (...),  k = x / w + cu,
// with r0 centred on the detector (so x/w is small near the centre) and the
// whole matrix divided by SID, so that w = L / SID and omega = w^-wexp.
// The FP64 map travels as FP32 pairs (hi + lo): each block evaluates it in
// float-float arithmetic at its tile's centre (the anchor), and its voxels
// take FP32 offsets from there (see BP3DAnchor).
struct BP2DParams {
    int nx, ny, nu, n_views, view0, views_total;
    int wexp;
    int parallel;              // w == 1 exactly
    float cu, scale;
    float m[kMaxViewsBP2D][6];   // x row (3), w row (3)
    float mlo[kMaxViewsBP2D][6]; // FP64 map - m
};

struct BP3DParams {
    int nx, ny, nz, nu, nv, n_views, view0, views_total;
    int wexp;
    int z_invariant;           // P[0][2] == P[2][2] == 0 for every view
    int accumulate;            // add into the output (view chunks after the first)
    float cu, cv, scale;
    float P[kMaxViewsConeBP][12];
    float Plo[kMaxViewsConeBP][12];  // FP64 map - P
};

// One view's map around a block's anchor A (the centre of its voxel tile),
// for a voxel at A + d:
//   u = cu + fu + (au . d) / (wa + w . d),   l = cl + fl + (al . d) / (wa + w . d)
// with the anchor's detector position cu + fu, cl + fl split into an
// integer and a fraction in [0, 1) (evaluated in float-float), au = r0 -
// (u_A - cu) r2 and al = r1 - (l_A - cv) r2.  |d| stays within the tile, so
// every FP32 term is small and the detector coordinate keeps ~1e-6 pixel
// where an absolute FP32 coordinate near pixel 300 carries ~2e-5.  bx, by:
// the TMA box origin of the tile (the TMA kernel stores cu, cl relative to it).
// The fields a circular-trajectory (z-invariant) kernel reads come first, in
// three 16-byte groups; w2, au2 (zero there) and the box origin follow.
struct __align__(16) BP3DAnchor {
    int cu, cl;
    float fu, fl;
    float wa, w0, w1, al2;
    float au0, au1, al0, al1;
    float w2, au2;
    int bx, by;
};

struct __align__(16) BP2DAnchor {
    int cu;
    float fu, wa, w0, w1, a0, a1, pad;
};

// ----------------------------------------------------- weights / filter --
struct WeightParams {
    int nu, nv, n_views;
    int cosine, redund;        // pyro_redund
    float su, sv, cu, cv, sdd;
    float delta;               // Parker half fan angle, or (range - pi) / 2 for PYRO_REDUND_SCAN
};

struct BetaTable {             // b_j - b_0 per view, for Parker weights
    float beta[kMaxViews2D];
};

struct FilterParams {
    long n_rows;
    int nu, pn, log2pn;
    int rows_per_view;         // rows of one view (nv for cone, 1 for 2D)
    int n_views;
    int apply_weights;         // fuse W_red W_cos into the load
    WeightParams w;
    float K[kMaxPadLength / 2 + 1];
};

// --------------------------------------------------------------- launchers --
// All launchers return cudaSuccess or the launch error; T is the storage type.
cudaError_t launch_fp2d(const void *vol, const void *volT, void *sino, int batch, const FP2DParams &p, pyro_dtype dt,
                        cudaStream_t s);
cudaError_t launch_transpose2d(const void *in, void *out, int batch, int nx, int ny, pyro_dtype dt, cudaStream_t s);
cudaError_t launch_bp3d_tex(cudaTextureObject_t tex, void *vol, const BP3DParams &p, pyro_dtype vol_dt, cudaStream_t s);
cudaError_t launch_fp3d_tex(cudaTextureObject_t tex, void *sino, const FP3DParams &p, pyro_dtype dt, cudaStream_t s);
cudaError_t launch_fp2d_adjoint(const void *sino, void *vol, void *volT, int batch, const FP2DParams &p,
                                cudaStream_t s);
cudaError_t launch_add_transposed(const void *accT, void *vol, int batch, int nx, int ny, cudaStream_t s);
cudaError_t launch_fp3d(const void *vol, void *sino, int batch, const FP3DParams &p, pyro_dtype dt,
                        cudaStream_t s);
cudaError_t launch_fp3d_adjoint(const void *sino, void *vol, int batch, const FP3DParams &p, cudaStream_t s);
// [z][y][x] -> [y][x][z] copy of one volume
cudaError_t launch_relayout_zmajor(const void *vol, void *vz, int nx, int ny, int nz, pyro_dtype dt, cudaStream_t s);
// the padded copy of the column kernels: storage FP32 / FP16 / BF16 (a
// half-size copy of an FP32 volume allowed); the sinogram FP32 or the storage type
cudaError_t launch_relayout_quad(const void *vol, void *vp, int nx, int ny, int nz, pyro_dtype dt,
                                   pyro_dtype storage, cudaStream_t s);
cudaError_t launch_fp3d_column(const void *vp, void *sino, int b, const FP3DParams &p, pyro_dtype storage,
                               pyro_dtype sino_dt, cudaStream_t s);
// forward projection of batch item b from its z-major copy; `sino` is the whole
// [batch][views_total][nv][nu] sinogram
cudaError_t launch_fp3d_zmajor(const void *vz, void *sino, int b, const FP3DParams &p, pyro_dtype dt,
                               cudaStream_t s);

// sino_dtype / vol_dtype may differ (FDK reads an FP32 workspace)
cudaError_t launch_bp2d(const void *sino, void *vol, int batch, const BP2DParams &p, pyro_dtype sino_dt,
                        pyro_dtype vol_dt, int accumulate, cudaStream_t s);
cudaError_t launch_bp2d_transpose(const void *vol, void *sino, int batch, const BP2DParams &p, cudaStream_t s);
cudaError_t launch_bp3d(const void *sino, void *vol, int batch, const BP3DParams &p, pyro_dtype sino_dt,
                        pyro_dtype vol_dt, cudaStream_t s);
cudaError_t launch_bp3d_transpose(const void *vol, void *sino, int batch, const BP3DParams &p, cudaStream_t s);
// TMA-staged cone BP: the sinogram as a 3D tensor map [batch * views][nv][nu],
// detector boxes of bu x bv elements (bu, the box width, is also the box's
// row pitch in shared memory: 80 or 144 floats, 96 or 160 halves); each of
// the kBPTmaStages ring stages holds the boxes of per_stage (1 or 2)
// consecutive views; a thread owns tile_z (8 or 16) voxels along z
constexpr int kBPTmaStages = 3;
struct BPTmaPlan {
    int tile_z, bu, bv, per_stage;
};
int tma_box_elems(int bu, int bv, size_t elem);  // one box, padded to 128 bytes
size_t bp3d_tma_smem_bytes(int n_views, int bu, int bv, size_t elem, int per_stage);
cudaError_t launch_bp3d_tma(const CUtensorMap &map, void *vol, int batch, const BP3DParams &p, const BPTmaPlan &pl,
                            pyro_dtype sino_dt, pyro_dtype vol_dt, cudaStream_t s);
// gathered cone adjoint: the weighted transposed sinogram yT[v][k][l] =
// dt |g| y[v][l][k] of batch item b for the chunk's views, then the gather
size_t gather_smem_bytes(const GatherParams &g);
cudaError_t launch_weighted_transpose(const void *sino, void *yT, int b, const FP3DParams &p, cudaStream_t s);
cudaError_t launch_gather_adjoint(const void *yT, void *vol, const GatherParams &g, int *status,
                                  cudaStream_t s);
// address of the device word a bounded wait sets when it gives up
cudaError_t status_word(int **ptr);
cudaError_t launch_wait_timeout_probe(unsigned long long limit_ns, cudaStream_t s);

cudaError_t launch_gather_probe(const void *buf, unsigned n16, int loads, unsigned *sink, long threads,
                                cudaStream_t s);
cudaError_t launch_bb_dots(const float *x, const float *xp, const float *g, const float *gp, long n, float *dots,
                           cudaStream_t s);
cudaError_t launch_bb_update(float *x, float *xp, const float *g, float *gp, long n, const float *dots, float alpha0,
                             float alpha_max, int first, float *alpha_out, cudaStream_t s);
cudaError_t launch_weights_table(void *sino, int batch, const WeightParams &w, const float *table, pyro_dtype dt,
                                 cudaStream_t s);
cudaError_t launch_redundancy_grad(const float *a, const float *g, float *out, int batch, int n_views, int nv, int nu,
                                   cudaStream_t s);
cudaError_t launch_weights(void *sino, int batch, const WeightParams &w, const BetaTable &beta, pyro_dtype dt,
                           cudaStream_t s);
// rows in (dtype in_dt) -> rows out (dtype out_dt); custom_K overrides p.K when non-null
cudaError_t launch_filter(const void *in, void *out, const FilterParams &p, const BetaTable *beta,
                          const float *custom_K, pyro_dtype in_dt, pyro_dtype out_dt, cudaStream_t s);
cudaError_t launch_filter_grad_K(const float *p, const float *g, float *dK, long n_rows, int nu, int pn,
                                 int log2pn, cudaStream_t s);

cudaError_t launch_tv(const float *x, float *grad, const float *base, float alpha, float lambda, float *value,
                      int batch, int nz, int ny, int nx, float eps, cudaStream_t s);
cudaError_t launch_axpby(const float *x, float *y, long n, float a, float b, cudaStream_t s);
cudaError_t launch_dot(const float *a, const float *b, long n, float *out, cudaStream_t s);

// residual CNN (kernels_cnn.cu)
bool conv_supported(int cin, int cout);
cudaError_t launch_conv3d(const void *X, const void *W, const float *bias, void *Y, int B, int D, int H, int Wd,
                          int cin, int cout, int relu, cudaStream_t s);
cudaError_t launch_conv3d_wgrad(const void *X, const void *dY, float *dW, int B, int D, int H, int Wd, int cin,
                                int cout, cudaStream_t s);
cudaError_t launch_weight_flip(const void *W, void *Wf, int cin, int cout, cudaStream_t s);
cudaError_t launch_cnn_elementwise(int op, const void *a, const void *b, void *y, const float *f, long n, int D,
                                   int H, int W, int C, cudaStream_t s);
cudaError_t launch_bias_grad(const void *dy, float *db, long nvox, int C, cudaStream_t s);
cudaError_t launch_mse(const float *out, const float *target, void *grad, float *loss, long n, cudaStream_t s);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, void *p16, long n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t s);

int device_sm_count();

// record the thread-local message returned by pyro_last_error()
void set_last_error(const char *fmt, ...);

}  // namespace pyro
