/*
 * pyro.h -- C ABI of the GB300-native known-operator CT layers.
 *
 * Re-implements the data-parallel hot path of PYRO-NN (Syben et al. 2019):
 * ray-driven forward projection, voxel-driven back-projection, their exact
 * transposes, cosine / Parker weights, ramp-type row filtering and FBP/FDK,
 * for 2D parallel-beam, 2D fan-beam and 3D cone-beam circular geometries.
 *
 * Common rules for every entry point
 * ----------------------------------
 *  Pointers.   Volume, sinogram, filter and workspace pointers are DEVICE
 *              pointers owned by the caller (16-byte aligned).  Geometry
 *              structs and the arrays they point to (angles, projection
 *              matrices) are HOST memory, read during the call only.
 *  Layout.     Volumes are [batch][nz][ny][nx] (2D: [batch][ny][nx]),
 *              x fastest.  Sinograms are [batch][n_views][nv][nu]
 *              (2D: [batch][n_views][nu]), u fastest.  Outputs are
 *              overwritten, never accumulated into.
 *  Geometry.   Voxel centre X_i = (i - (N-1)/2) * s (volume centred on the
 *              iso-centre).  Detector coordinate u_k = (k - (nu-1)/2) * su.
 *              View j: central ray c = (cos b_j, sin b_j, 0), detector axis
 *              e_u = (-sin b_j, cos b_j, 0), e_v = (0, 0, 1).  Fan/cone
 *              source S = -SID c, flat detector at distance SDD from S.
 *              Cone-beam views are 3x4 projection matrices P with
 *              (x, y, w) = P (X, 1) and detector index (x/w, y/w)
 *              (Section "Trajectories"); NULL means the circular
 *              trajectory P = K [R | -R S], R = [e_u; e_v; c],
 *              K = [[SDD/su, 0, (nu-1)/2], [0, SDD/sv, (nv-1)/2], [0, 0, 1]].
 *  Interpolation. Bi-/trilinear over the zero-extended arrays (values
 *              outside the array are 0), computed in FP32 in software.
 *  Precision.  dtype selects the STORAGE type of volumes and sinograms;
 *              arithmetic and accumulation are always FP32.
 *  Execution.  Every call is asynchronous on `stream` (a cudaStream_t;
 *              NULL = legacy default stream) and uses the current device.
 *              Host-side argument errors return PYRO_EINVAL before anything
 *              is enqueued; launch failures return PYRO_ECUDA.  The library
 *              makes no device allocation: scratch comes from the caller's
 *              workspace arguments (pyro_fdk_noalloc alone uses a static
 *              array of the library).  On a non-zero return,
 *              pyro_last_error() gives a message (thread-local).
 */
#ifndef PYRO_H
#define PYRO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PYRO_API __attribute__((visibility("default")))

typedef enum {
    PYRO_OK = 0,
    PYRO_EINVAL = 1,       /* invalid argument or geometry                  */
    PYRO_ECUDA = 2,        /* a CUDA launch or runtime call failed          */
    PYRO_ETIMEOUT = 3,     /* a bounded device-side wait gave up            */
    PYRO_EUNSUPPORTED = 4, /* valid request this build does not implement   */
    PYRO_EWORKSPACE = 5    /* workspace missing or smaller than required    */
} pyro_status;

typedef enum { PYRO_F32 = 0, PYRO_F16 = 1, PYRO_BF16 = 2 } pyro_dtype;

/* voxel weight of the back-projectors: omega = 1, SID/L or (SID/L)^2 with
 * L the depth of the voxel from the source along the central ray */
typedef enum { PYRO_W_NONE = 0, PYRO_W_INV_L = 1, PYRO_W_INV_L2 = 2 } pyro_bp_weight;

typedef enum { PYRO_RAMLAK = 0, PYRO_RAMP = 1, PYRO_SHEPP_LOGAN = 2, PYRO_FILTER_CUSTOM = 3 } pyro_filter;

/* redundancy weight W_red: 1/2 (full 360 degree scan), Parker short scan
 * (pi + 2 delta), 1, or PYRO_REDUND_SCAN: the weighting for a scan over the
 * geometry's `range` R, 0 < R <= 2 pi (super-short scans, R < pi + 2 delta,
 * named in Section "Geometric Correction Weights", as well as short and
 * over-scans): Parker's form with delta replaced by (R - pi) / 2.  The rays
 * whose line the scan measures twice get smooth weights that add to 1 over
 * the two measurements, the rays measured once get 1. */
typedef enum {
    PYRO_REDUND_FULL = 0,
    PYRO_REDUND_PARKER = 1,
    PYRO_REDUND_NONE = 2,
    PYRO_REDUND_SCAN = 3
} pyro_redund;

/* 2D parallel / fan geometry (Section "Reconstruction & Geometry": volume
 * shape and spacing, detector shape and spacing, number of projections,
 * angular range, SID and SDD, plus one central-ray direction per view). */
typedef struct {
    int nx, ny;            /* image shape                                    */
    double sx, sy;         /* pixel spacing, mm                              */
    int nu;                /* detector bins                                  */
    double su;             /* bin spacing, mm                                */
    int n_views;           /* number of projections                          */
    const double *angles;  /* [n_views] view angles b_j (rad), or NULL:      */
                           /*   b_j = j * range / n_views                    */
    double range;          /* angular range, rad                             */
    double sid, sdd;       /* fan beam only: source-iso / source-detector mm */
    double step;           /* FP sample step along the ray, mm; <= 0: half   */
                           /*   the smallest pixel spacing                   */
} pyro_geom2d;

/* 3D cone-beam geometry (same attributes; trajectory as projection matrices) */
typedef struct {
    int nx, ny, nz;
    double sx, sy, sz;
    int nu, nv;               /* detector columns (u) and rows (v)            */
    double su, sv;
    int n_views;
    const double *proj_mats;  /* [n_views][3][4] row-major, or NULL: circular */
    const double *angles;     /* [n_views] rad or NULL (j * range / n_views);  */
                              /*   used for circular matrices and for W_red    */
    double range, sid, sdd;
    double step;              /* as in pyro_geom2d                             */
} pyro_geom3d;

/* --- Ray-driven forward projection A (Section "The Operator as a Layer"). ---
 * One line integral per detector pixel.  The ray is X(w) = a + w g,
 * parametrised by the depth w along the view's principal axis (g has unit
 * depth; a is the bin position u e_u for parallel beam, the source
 * otherwise), and sampled on equally spaced depth planes:
 *   p = step |g| sum_{m=-M..M} f(a + (w0 + m step) g),
 * w0 the depth of the iso-centre (0 for parallel beam, SID otherwise),
 * M = ceil(T / step), T = half diagonal of the box (N+1)*s, f the
 * zero-extended interpolant.  vol [batch][...] -> sino [batch][...]. */
PYRO_API int pyro_fp_par2d(const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_dtype dtype,
                           void *stream);
PYRO_API int pyro_fp_fan2d(const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_dtype dtype,
                           void *stream);
PYRO_API int pyro_fp_cone3d(const void *vol, void *sino, int batch, const pyro_geom3d *g, pyro_dtype dtype,
                            void *stream);

/* --- The same 2D forward projections, also reading a transposed copy of
 * the batch kept in `workspace` (device, at least pyro_fp2d_workspace_bytes
 * bytes: batch images of `dtype`; PYRO_EWORKSPACE otherwise): a warp's lanes
 * take consecutive detector bins, and for views whose rays run closer to x
 * than to y the bins' taps are contiguous in the transposed copy.  Results
 * equal pyro_fp_par2d / pyro_fp_fan2d up to FP32 rounding order. */
PYRO_API size_t pyro_fp2d_workspace_bytes(const pyro_geom2d *g, int batch, pyro_dtype dtype);
PYRO_API int pyro_fp_par2d_ws(const void *vol, void *sino, int batch, const pyro_geom2d *g, void *workspace,
                              size_t workspace_bytes, pyro_dtype dtype, void *stream);
PYRO_API int pyro_fp_fan2d_ws(const void *vol, void *sino, int batch, const pyro_geom2d *g, void *workspace,
                              size_t workspace_bytes, pyro_dtype dtype, void *stream);
/* --- Texture mode (Section "The Operator as a Layer"): the paper's fast
 * forward- and back-projection modes, which keep a second copy of the data
 * in a CUDA array read with hardware filtering.  A texture is the one object
 * this library allocates; the caller owns it and releases it with
 * pyro_texture_destroy (NULL is accepted).
 *   pyro_texture_volume_create: a [nz][ny][nx] 3D array (trilinear filtering).
 *   pyro_texture_sinogram_create: a [n_views][nv][nu] layered 2D array, one
 *     layer per view (bilinear filtering).
 * Both hold PYRO_F32 or PYRO_F16 values (PYRO_EUNSUPPORTED otherwise), have
 * a zero border (the zero extension of the software path) and are refused
 * with PYRO_EINVAL beyond the device's texture limits.  pyro_texture_upload
 * copies a device buffer of the texture's dtype and extent into it on
 * `stream`.
 *   pyro_fp_cone3d_tex: FP of a volume texture (one volume, no batch) into
 *     `sino` [n_views][nv][nu] of `dtype` storage; same rays, sample grid and
 *     scaling as pyro_fp_cone3d.
 *   pyro_bp_cone3d_tex: voxel-driven BP of a sinogram texture into `vol`
 *     [nz][ny][nx] of `dtype` storage; same map, weights and scale as
 *     pyro_bp_cone3d.
 * The geometry's shapes must equal the texture's (PYRO_EINVAL).  The
 * hardware's interpolation weights are fixed point with 8 fractional bits,
 * so results differ from the FP32 software path by about 1e-4 .. 1e-3
 * relative. */
typedef struct pyro_texture_s *pyro_texture;
PYRO_API int pyro_texture_volume_create(int nx, int ny, int nz, pyro_dtype dtype, pyro_texture *out);
PYRO_API int pyro_texture_sinogram_create(int nu, int nv, int n_views, pyro_dtype dtype, pyro_texture *out);
PYRO_API int pyro_texture_upload(pyro_texture t, const void *src, void *stream);
PYRO_API int pyro_texture_destroy(pyro_texture t);
PYRO_API int pyro_fp_cone3d_tex(pyro_texture t, void *sino, const pyro_geom3d *g, pyro_dtype dtype, void *stream);
PYRO_API int pyro_bp_cone3d_tex(pyro_texture t, void *vol, const pyro_geom3d *g, pyro_bp_weight w, float scale,
                                pyro_dtype dtype, void *stream);

/* The exact adjoints of the 2D projections with a transposed FP32
 * accumulator in `workspace` (pyro_fp2d_workspace_bytes(g, batch, PYRO_F32)
 * bytes at least) for the views whose rays run closer to x, added back into
 * vol at the end.  Equal to pyro_fpT_par2d / pyro_fpT_fan2d up to FP32
 * summation order.  PYRO_F32 only. */
PYRO_API int pyro_fpT_par2d_ws(const void *sino, void *vol, int batch, const pyro_geom2d *g, void *workspace,
                               size_t workspace_bytes, pyro_dtype dtype, void *stream);
PYRO_API int pyro_fpT_fan2d_ws(const void *sino, void *vol, int batch, const pyro_geom2d *g, void *workspace,
                               size_t workspace_bytes, pyro_dtype dtype, void *stream);

/* --- The projection matrices the cone-beam calls use for geometry `g`
 * (the circular trajectory's when g->proj_mats is NULL, else the given
 * ones), normalised as the calls normalise them: third row (the depth) of
 * unit norm in its first three entries, positive depth at the iso-centre.
 * out: HOST array [n_views][3][4] (row-major doubles) owned by the caller.
 * Host-only (no device work): lets a caller hand a subset of views, or
 * matrices shifted to a sub-volume, back to the calls as proj_mats. */
PYRO_API int pyro_cone_projection_matrices(const pyro_geom3d *g, double *out);

/* --- The same cone-beam forward projection, computed from a copy of the
 * volume re-laid out z-fastest in `workspace` (device, at least
 * pyro_fp_cone3d_workspace_bytes bytes; PYRO_EWORKSPACE otherwise).  For
 * circular-type trajectories the copy is a quad copy: the volume padded by
 * two voxels before and after the data in x and y and one in z, each cell
 * (x, y, z) holding the four voxels (x, y), (x + 1, y), (x, y + 1),
 * (x + 1, y + 1) at z, i.e. 4 (nx + 4)(ny + 4)(nz + 2) elements of `dtype`;
 * other trajectories use the first nx ny nz of them.  This is the
 * memory-for-speed trade the paper describes for its texture mode (the
 * volume is held again, Section "The Operator as a Layer"); pyro_fp_cone3d
 * is the memory-lean mode.  Results are identical up to FP32 summation
 * order; the workspace is scratch. */
PYRO_API size_t pyro_fp_cone3d_workspace_bytes(const pyro_geom3d *g, pyro_dtype dtype);
PYRO_API int pyro_fp_cone3d_ws(const void *vol, void *sino, int batch, const pyro_geom3d *g, void *workspace,
                               size_t workspace_bytes, pyro_dtype dtype, void *stream);

/* --- The same staged forward projection with the workspace copy held in
 * `storage` while the volume and the sinogram stay in `dtype`: an FP32
 * volume projected from an FP16 or BF16 copy (half the workspace; the
 * volume's values rounded to 16 bits, accumulation along the rays in FP32,
 * an FP32 sinogram), a half-storage copy of an FP32 iterate (Section "The
 * Operator as a Layer": the copy is the paper's memory-for-speed trade).  storage == dtype is pyro_fp_cone3d_ws.  The
 * workspace needs pyro_fp_cone3d_workspace_bytes(g, storage) bytes.
 * PYRO_EUNSUPPORTED for storage != dtype with a non-FP32 volume or a
 * trajectory other than circular-type (detector v axis along z). */
PYRO_API int pyro_fp_cone3d_ws_storage(const void *vol, void *sino, int batch, const pyro_geom3d *g, void *workspace,
                                       size_t workspace_bytes, pyro_dtype dtype, pyro_dtype storage, void *stream);

/* --- Exact adjoint A^T of the forward projectors (the gradient of the FP
 * layer, Section "The Known Operator": the gradient of A is A^T).  Scatters
 * step * y * (interpolation weights) into the volume with FP32 atomics, so
 * results agree with the sequential sum to rounding, not bit for bit.
 * sino [batch][...] -> vol [batch][...].  Only PYRO_F32 is supported. */
PYRO_API int pyro_fpT_par2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_dtype dtype,
                            void *stream);
PYRO_API int pyro_fpT_fan2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_dtype dtype,
                            void *stream);
PYRO_API int pyro_fpT_cone3d(const void *sino, void *vol, int batch, const pyro_geom3d *g, pyro_dtype dtype,
                             void *stream);

/* --- The same exact adjoint of the cone-beam projector, gathered voxel by
 * voxel for circular-type trajectories (the detector's v axis along the
 * volume's z axis): the ray-weighted sinogram is transposed into
 * `workspace` (device, at least pyro_fpT_cone3d_workspace_bytes bytes, one
 * view x nu x nv FP32 sinogram; PYRO_EWORKSPACE otherwise), then every
 * voxel sums the samples whose interpolation reaches it in a fixed order:
 * no atomics, and the result is the same bit for bit from run to run.
 * Other trajectories, and detectors whose rows are so fine that one voxel's
 * tent reaches more than 29 of them (a row step under 1/14.5 voxel on the
 * nearest plane), fall back to pyro_fpT_cone3d (the workspace is then
 * unused).  Results agree with it to FP32 rounding; the workspace is
 * scratch.  PYRO_F32 only.  pyro_sync_status reports PYRO_ECUDA if a
 * shared-memory table outgrew its host-computed bound (never expected). */
PYRO_API size_t pyro_fpT_cone3d_workspace_bytes(const pyro_geom3d *g);
PYRO_API int pyro_fpT_cone3d_ws(const void *sino, void *vol, int batch, const pyro_geom3d *g, void *workspace,
                                size_t workspace_bytes, pyro_dtype dtype, void *stream);

/* --- Voxel-driven back-projection (Section "The Operator as a Layer"; the
 * cone-beam form after Scherl et al. with projection matrices):
 *   x(X) = scale * sum_j omega_j(X) * L(y_j; k_j(X) [, l_j(X)]),
 * k_j(X) the detector index X projects to in view j, L linear (2D) or
 * bilinear (3D) interpolation of the zero-extended detector.
 * sino [batch][...] -> vol [batch][...]. */
PYRO_API int pyro_bp_par2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_bp_weight w,
                           float scale, pyro_dtype dtype, void *stream);
PYRO_API int pyro_bp_fan2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_bp_weight w,
                           float scale, pyro_dtype dtype, void *stream);
PYRO_API int pyro_bp_cone3d(const void *sino, void *vol, int batch, const pyro_geom3d *g, pyro_bp_weight w,
                            float scale, pyro_dtype dtype, void *stream);

/* --- Transpose of the voxel-driven back-projection (its autograd backward):
 * scatters scale * omega * (interpolation weights) * g(X) into the detector
 * with FP32 atomics.  vol [batch][...] -> sino [batch][...].  PYRO_F32 only. */
PYRO_API int pyro_bpT_par2d(const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_bp_weight w,
                            float scale, pyro_dtype dtype, void *stream);
PYRO_API int pyro_bpT_fan2d(const void *vol, void *sino, int batch, const pyro_geom2d *g, pyro_bp_weight w,
                            float scale, pyro_dtype dtype, void *stream);
PYRO_API int pyro_bpT_cone3d(const void *vol, void *sino, int batch, const pyro_geom3d *g, pyro_bp_weight w,
                             float scale, pyro_dtype dtype, void *stream);

/* --- Geometric correction weights, in place (Section "Geometric Correction
 * Weights", Eq. 5): p <- W_red W_cos p.  W_cos = SDD / sqrt(SDD^2+u^2+v^2)
 * when `cosine` != 0.  W_red per pyro_redund; Parker uses the half fan angle
 * delta = atan(nu su / (2 SDD)), gamma = atan(u / SDD) and b_j - b_0.
 * sino [batch][n_views][nu] (2D, v = 0) or [batch][n_views][nv][nu]. */
PYRO_API int pyro_weights2d(void *sino, int batch, const pyro_geom2d *g, int cosine, pyro_redund redund,
                            pyro_dtype dtype, void *stream);
PYRO_API int pyro_weights3d(void *sino, int batch, const pyro_geom3d *g, int cosine, pyro_redund redund,
                            pyro_dtype dtype, void *stream);

/* --- Row filtering F^H K F (Eq. 4; Section "Filters").  Each of n_rows rows
 * of nu samples is zero-padded to pn = smallest power of two >= 2 nu,
 * transformed, multiplied by the real even diagonal K[0..pn/2] and
 * transformed back; the first nu samples are kept.  Built-in K: Ram-Lak and
 * Shepp-Logan are the DFTs of tau * h(n), h the spatial kernels of Kak &
 * Slaney on sample spacing tau (this equals linear convolution with h);
 * ramp is K[m] = |m| / (pn tau).  PYRO_FILTER_CUSTOM reads K from the
 * DEVICE array custom_K[pn/2 + 1] (FP32).  in/out may alias.  FP32 FFT.
 * nu <= 4096. */
PYRO_API int pyro_filter_rows(const void *in, void *out, long n_rows, int nu, double tau, pyro_filter kind,
                              const float *custom_K, pyro_dtype dtype, void *stream);

/* padded length pn used by pyro_filter_rows for a row of nu samples */
/* --- Learnable redundancy weights (Section "Geometric Correction Weights":
 * the paper proposes learning W_red of Eq. 5 like the filter).
 * pyro_weights3d_table: sino [batch][V][nv][nu] *= (cosine ? W_cos : 1) *
 * table[view][k], in place; table is a DEVICE FP32 array [V][nu] owned by
 * the caller (one weight per view and detector column, as the short-scan
 * weights are).  pyro_redundancy_grad: out[view][k] = sum over the batch and
 * the rows of a * g (DEVICE FP32, [batch][V][nv][nu] each; out [V][nu]):
 * with a = W_cos p and g the filtered back-projected gradient (the filter
 * and the cosine weight are symmetric), the gradient of a loss with respect
 * to the table.  Errors as for pyro_weights3d. */
PYRO_API int pyro_weights3d_table(void *sino, int batch, const pyro_geom3d *g, const float *table, int cosine,
                                  pyro_dtype dtype, void *stream);
PYRO_API int pyro_redundancy_grad(const float *a, const float *g, float *out, int batch, int n_views, int nv, int nu,
                                  void *stream);

PYRO_API int pyro_filter_pad_length(int nu);

/* The diagonal K[0..pn/2] of a built-in filter (Ram-Lak, ramp or
 * Shepp-Logan on sample spacing tau), written to the HOST array K_out of
 * pn/2 + 1 floats: the initial value of a learnable filter (Eq. 6). */
PYRO_API int pyro_filter_spectrum(pyro_filter kind, int nu, double tau, float *K_out);

/* --- Gradient of a loss with respect to a custom K (Eq. 6, filter learning):
 * dK[m] = sum_rows c_m / pn * Re(P[m] conj(G[m])), P and G the length-pn
 * DFTs of the zero-padded rows of p (the filter's input) and g (dL/dq),
 * c_m = 1 for m in {0, pn/2} and 2 otherwise.  FP32 device arrays:
 * p, g [n_rows][nu], dK [pn/2 + 1] (overwritten). */
PYRO_API int pyro_filter_grad_K(const float *p, const float *g, float *dK, long n_rows, int nu, void *stream);

/* --- FBP / FDK (Eq. 4, Eq. 5): x = A_bp F^H K F W_red W_cos p.
 * Cone: tau = su * SID / SDD (virtual detector at the iso-centre),
 *       omega = (SID / L)^2, scale = range / n_views (Feldkamp).
 * Fan:  the same with v = 0.
 * Parallel: no weights, tau = su, scale = pi / n_views.
 * The weighted, filtered sinogram is kept in `workspace` (device, at least
 * pyro_*_workspace_bytes bytes; PYRO_EWORKSPACE otherwise). */
PYRO_API size_t pyro_fdk_workspace_bytes(const pyro_geom3d *g, int batch);
PYRO_API int pyro_fdk(const void *sino, void *vol, int batch, const pyro_geom3d *g, pyro_filter kind,
                      const float *custom_K, pyro_redund redund, void *workspace, size_t workspace_bytes,
                      pyro_dtype dtype, void *stream);
PYRO_API size_t pyro_fbp2d_workspace_bytes(const pyro_geom2d *g, int batch);
PYRO_API int pyro_fbp_par2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_filter kind,
                            const float *custom_K, void *workspace, size_t workspace_bytes, pyro_dtype dtype,
                            void *stream);
PYRO_API int pyro_fbp_fan2d(const void *sino, void *vol, int batch, const pyro_geom2d *g, pyro_filter kind,
                            const float *custom_K, pyro_redund redund, void *workspace, size_t workspace_bytes,
                            pyro_dtype dtype, void *stream);

/* --- Total variation for the iterative reconstruction of Eq. 7
 * (min |A x - p|^2 + lambda TV(x)), in the smoothed anisotropic form
 *   TV(x) = sum_{axes a} sum_i phi(x_{i+e_a} - x_i),  phi(d) = sqrt(d^2+eps^2) - eps,
 * over the forward differences that stay inside the volume.  FP32 device
 * arrays [batch][nz][ny][nx].  grad (may be NULL) receives
 * alpha * base + lambda * dTV/dx (base may be NULL = 0 and may alias grad);
 * value (may be NULL) receives TV(x) per batch item, reduced in FP32
 * (block sums, then FP32 atomics: not bit-reproducible across runs). */
PYRO_API int pyro_tv(const float *x, float *grad, const float *base, float alpha, float lambda, float *value,
                     int batch, int nz, int ny, int nx, float eps, void *stream);
/* y = a x + b y over n FP32 device values (the gradient step of Eq. 7) */
PYRO_API int pyro_axpby(const float *x, float *y, long n, float a, float b, void *stream);
/* out[0] = sum a_i b_i over n FP32 device values; out is a DEVICE float,
 * reduced in FP32 (block sums, then FP32 atomics) */
PYRO_API int pyro_dot(const float *a, const float *b, long n, float *out, void *stream);
/* --- The Barzilai-Borwein step of the iteration, kept on the device (no
 * host read of a scalar, so that an iteration can be captured in a CUDA
 * graph).  pyro_bb_dots: dots[0] = |x - x_prev|^2, dots[1] =
 * (x - x_prev).(g - g_prev) (DEVICE float[2], overwritten; FP32 reduction).
 * pyro_bb_update: alpha = alpha0 when `first` (or when dots[1] <= 0), else
 * dots[0] / dots[1] clamped to [0, alpha_max]; then x_prev = x, g_prev = g,
 * x -= alpha g over n FP32 device values; alpha_out (DEVICE float, may be
 * NULL) receives the alpha used. */
PYRO_API int pyro_bb_dots(const float *x, const float *x_prev, const float *g, const float *g_prev, long n,
                          float *dots, void *stream);
PYRO_API int pyro_bb_update(float *x, float *x_prev, const float *g, float *g_prev, long n, const float *dots,
                            float alpha0, float alpha_max, int first, float *alpha_out, void *stream);

/* --- Residual 3D CNN used as a learned initialiser of the iterative
 * reconstruction.  The paper has no network of its own; its "learned parts"
 * outlook (Section "Network Architectures") is met by this small BF16
 * network trained with the library's operators.  Activations are
 * channels-last BF16 [batch][nz][ny][nx][c]; weights are BF16
 * [27][cout][cin] (tap = (dz*3+dy)*3+dx of a 3x3x3 window, stride 1, zero
 * padding 1); bias, gradients of weights and biases are FP32.  Supported
 * (cin, cout): both in {16, 32, 64} (5th-generation tensor cores, tcgen05,
 * bf16 -> fp32 in tensor memory), or (1, 16) / (16, 1) (CUDA cores).  The tensor-core shapes work on
 * blocks of 128 voxels TX x TY x TZ with TX = min(nx, 64),
 * TY = min(ny, 128 / TX), TZ = 128 / (TX TY): nx must be 8, 16, 32 or a
 * multiple of 64, and ny, nz must be multiples of TY, TZ.
 * pyro_conv3d:        y = [relu](conv(x, w) + bias), bias may be NULL.
 * pyro_conv3d_wgrad:  dw[tap][co][ci] = sum_v dy[v][co] x[v + tap][ci]
 *                     (overwritten; FP32 atomics across blocks).
 * pyro_conv3d_flip_weights: wf[t][ci][co] = w[26 - t][co][ci], the weights
 *                     of the data gradient dx = conv(dy, wf) (cin <-> cout). */
PYRO_API int pyro_conv3d(const void *x, const void *w, const float *bias, void *y, int batch, int nz, int ny, int nx,
                         int cin, int cout, int relu, void *stream);
PYRO_API int pyro_conv3d_wgrad(const void *x, const void *dy, float *dw, int batch, int nz, int ny, int nx, int cin,
                               int cout, void *stream);
PYRO_API int pyro_conv3d_flip_weights(const void *w, void *wf, int cin, int cout, void *stream);

/* elementwise steps of the network; n = number of elements WRITTEN to y.
 * (nz, ny, nx) are the full-resolution dims for AVGPOOL2 and AVGPOOL2_BWD,
 * and the half-resolution dims for UPSAMPLE2 and UPSAMPLE2_BWD. */
typedef enum {
    PYRO_CNN_RELU_BWD = 0,     /* y(bf16 grad, in place) *= (a(bf16 activation) > 0)      */
    PYRO_CNN_AVGPOOL2 = 1,     /* y = 2x2x2 mean of a                                     */
    PYRO_CNN_AVGPOOL2_BWD = 2, /* y = a(upper level) / 8 spread over the 8 children       */
    PYRO_CNN_UPSAMPLE2 = 3,    /* y = nearest 2x upsampling of a, plus b (skip) if b != 0 */
    PYRO_CNN_UPSAMPLE2_BWD = 4,/* y = sum of a over the 8 children                        */
    PYRO_CNN_ADD = 5,          /* y = a + b (bf16)                                        */
    PYRO_CNN_F32_TO_BF16 = 6,  /* y(bf16) = a(f32)                                        */
    PYRO_CNN_BF16_TO_F32 = 7,  /* y(f32) = a(bf16)                                        */
    PYRO_CNN_RESIDUAL = 8      /* y(f32) = f(f32) + a(bf16)                               */
} pyro_cnn_op_kind;
PYRO_API int pyro_cnn_op(int op, const void *a, const void *b, void *y, const float *f, long n, int nz, int ny, int nx,
                         int c, void *stream);
/* db[c] = sum over nvox voxels of dy[v][c] (dy bf16 channels-last, db FP32, overwritten) */
PYRO_API int pyro_cnn_bias_grad(const void *dy, float *db, long nvox, int c, void *stream);
/* loss[0] = mean (out - target)^2 (FP32, device); grad (bf16, may be NULL) = 2 (out - target) / n */
PYRO_API int pyro_cnn_mse(const float *out, const float *target, void *grad, float *loss, long n, void *stream);
/* Adam step on FP32 master parameters p with gradient g and moments m, v
 * (step counts from 1); p16 (may be NULL) receives the bf16 copy of p. */
PYRO_API int pyro_cnn_adam(float *p, const float *g, float *m, float *v, void *p16, long n, float lr, float beta1,
                           float beta2, float eps, int step, void *stream);

/* --- FDK without any device allocation by the caller.  The paper has no
 * counterpart: this serves callers that only hold the input and output
 * buffers and cannot allocate device memory (e.g. a reconstruction stage
 * inside an acquisition pipeline, or a host application whose allocator owns
 * all device memory), so they cannot pass the workspace pyro_fdk needs.
 * Same arguments and result as pyro_fdk, minus the workspace: the scratch is
 * a static device array of PYRO_FDK_NOALLOC_SCRATCH_BYTES (64 MiB) inside the
 * library, held on every GPU that loads it until the process exits.
 * Problems needing more (4 * batch * n_views * nv * nu bytes) return
 * PYRO_EWORKSPACE.  The first call on a device looks up the array's address
 * (and again the first call in a new context on it, e.g. after a
 * cudaDeviceReset); that first call should come before any stream capture
 * on that device.  All calls on a
 * device share the array (it keeps the last call's contents): calls that
 * overlap on the GPU race with each other.  No allocation is made. */
#define PYRO_FDK_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
PYRO_API int pyro_fdk_noalloc(const void *sino, void *vol, int batch, const pyro_geom3d *g, pyro_filter kind,
                              const float *custom_K, pyro_redund redund, pyro_dtype dtype, void *stream);

/* thread-local message describing the last non-OK status of this thread */
/* --- Waits for the stream and reports what happened on it: PYRO_OK,
 * PYRO_ECUDA with the CUDA error's text in pyro_last_error, or PYRO_ETIMEOUT
 * when a bounded device-side wait gave up (the TMA-staged cone BP waits on
 * its copies with an iteration limit; a block that gives up sets a device
 * status word, which this call reads and clears).  Synchronous. */
PYRO_API int pyro_sync_status(void *stream);
/* --- Self-test of that path (no counterpart in the paper): enqueues a kernel
 * whose single warp waits on a barrier that nothing completes, gives up after
 * limit_ms (1..1000) milliseconds and sets the status word, so that the next
 * pyro_sync_status returns PYRO_ETIMEOUT.  Nothing faults and nothing hangs;
 * the context stays usable. */
PYRO_API int pyro_selftest_wait_timeout(int limit_ms, void *stream);

/* --- Gather-bandwidth probe (no counterpart in the paper; the roofline
 * denominator for gather-bound kernels): `threads` threads each read
 * loads_per_thread 16-byte chunks at pseudo-random positions of the DEVICE
 * buffer `buf` (bytes, 16-byte aligned; a buffer smaller than L2 measures
 * L2 gathers).  sink: DEVICE array of 1024 unsigned, written only to keep
 * the loads alive.  Time it with events on `stream`: bandwidth =
 * 16 * threads * loads_per_thread / time. */
PYRO_API int pyro_probe_gather(const void *buf, size_t bytes, int loads_per_thread, long threads, unsigned *sink,
                               void *stream);
PYRO_API const char *pyro_last_error(void);
/* library version string */
PYRO_API const char *pyro_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PYRO_H */
