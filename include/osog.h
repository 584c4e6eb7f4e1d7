/*
 * osog.h - C ABI of libosog, a GB300 (sm_103a) renderer for the OSOG
 * optical forward model (arxiv 2606.21381).
 *
 * The library computes, for a structure-of-arrays tensor of transparent
 * particles, the multi-modal micrograph f(Theta) = I of Sec. III:
 *
 *   1. per-pixel thickness footprints of ellipsoids and bevelled prisms
 *      (Sec. III.A; the prism is the half-space intersection of Eq. 1);
 *   2. composition of the optical path difference OPD = sum_p dn_p t_p and
 *      of the absorption exponent ATT = sum_p mu_p t_p, overlaps adding
 *      (Eq. 2's integral over z, Eq. 7's accumulate=True splat);
 *   3. the exit wave E = exp(-ATT) exp(i 2 pi OPD / lambda) (Eq. 2, with the
 *      Beer-Lambert amplitude of Eq. 4);
 *   4. the optical head: forward 2-D DFT, multiplication by the transfer
 *      function of each selected modality (pupil of Eq. 3 with NA cutoff and
 *      defocus; oblique illumination as the pupil shifted by k_ill; DIC as
 *      the coherent shear difference of Eq. 5), inverse 2-D DFT;
 *   5. intensity I = |E_out|^2 (Sec. III.B, "I_BF = |U_exit * h_obj|^2").
 *
 * Conventions shared by every entry point:
 *   - Particle tensor: float32, planar [9][ld] on the device, rows
 *       0 cx (px)  1 cy (px)  2 theta (rad, from +x toward +y)
 *       3 a | hx (px)  4 b | hy (px)  5 T (um)  6 dn  7 mu (1/um)
 *       8 kind (0 = ellipsoid with semi-axes a, b and full thickness T;
 *               1 = rectangular prism with half-lengths hx, hy, thickness T
 *               and chamfers of slope bevel_slope on all top/bottom edges;
 *               2 = general convex polyhedron, osog_render_polyhedra only).
 *   - Pixel (i, j) is sampled at its centre (x, y) = (j + 0.5, i + 0.5) px;
 *     rows are y.  Images are float32 [K][H][W], K = number of bits set in
 *     optics->modes, in bit order brightfield, oblique, DIC.
 *   - H and W are powers of two in [32, 2048] (OSOG_ERR_UNSUPPORTED_SIZE).
 *   - All device buffers belong to the caller.  The library allocates device
 *     memory only in osog_plan_create; every other call runs asynchronously
 *     on the given stream and allocates nothing.
 *   - Errors found on the host are returned at once (and described by
 *     osog_last_error).  Errors found on the device (non-finite or invalid
 *     particle fields, bin overflow, timeouts) are latched in the plan's
 *     device status word; osog_sync_status synchronises the stream, returns
 *     the first latched code and clears it.  Nothing aborts, traps or prints.
 *   - A plan may be used by one host thread at a time.
 */
#ifndef OSOG_H
#define OSOG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define OSOG_OK 0
#define OSOG_ERR_INVALID_ARG 1        /* bad pointer, size or option */
#define OSOG_ERR_UNSUPPORTED_SIZE 2   /* H or W not a power of two in [32, 2048] */
#define OSOG_ERR_WORKSPACE 3          /* workspace too small or misaligned */
#define OSOG_ERR_BIN_OVERFLOW 4       /* more particle-band pairs than reserved */
#define OSOG_ERR_NONFINITE_INPUT 5    /* NaN or Inf in a particle field */
#define OSOG_ERR_TIMEOUT 6            /* a bounded device wait gave up */
#define OSOG_ERR_CUDA 7               /* a CUDA runtime call failed */
#define OSOG_ERR_INVALID_PARTICLE 8   /* a <= 0, b <= 0, T < 0, unknown kind, or a
                                         kind-2 particle without a valid plane range */

/* Modality bits of osog_optics_t.modes. */
#define OSOG_MODE_BRIGHTFIELD 1u
#define OSOG_MODE_OBLIQUE 2u
#define OSOG_MODE_DIC 4u

/* Kernel classes reported by osog_profile_end. */
#define OSOG_KERNEL_BIN_COUNT 0
#define OSOG_KERNEL_BIN_SCAN 1
#define OSOG_KERNEL_BIN_FILL 2
#define OSOG_KERNEL_STRIP_FORWARD 3
#define OSOG_KERNEL_COLUMN 4
#define OSOG_KERNEL_STRIP_INVERSE 5
#define OSOG_KERNEL_BWD_ROWS 6
#define OSOG_KERNEL_BWD_COLUMN 7
#define OSOG_KERNEL_BWD_STRIP 8
#define OSOG_KERNEL_BWD_REDUCE 9
#define OSOG_KERNEL_PERSISTENT 10
#define OSOG_KERNEL_RASTER 11
#define OSOG_KERNEL_CLASS_COUNT 12

typedef struct osog_plan osog_plan_t;
/* Binary-compatible with cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *osog_stream_t;

/*
 * Optics of one scene (host struct, passed by pointer; Sec. III.B).
 *   dx_um       pixel pitch in the sample plane (um)
 *   lambda_um   wavelength (um)
 *   NA          numerical aperture; k_NA = 2 pi NA / lambda (Eq. 3)
 *   n_medium    medium index n_m; k0 = 2 pi n_m / lambda (Eq. 2, Eq. 3)
 *   defocus_um  dz of Eq. 3; the pupil phase is dz (sqrt(k0^2-|k|^2) - k0)
 *   modes       OSOG_MODE_* bits; K = number of bits set (1..3)
 *   oblique_frac, oblique_angle
 *               oblique modality: transfer P(k + k_ill) with
 *               k_ill = oblique_frac k_NA (cos, sin)(oblique_angle)
 *   shear_px, shear_angle, bias_phase
 *               DIC (Eq. 5): shear distance 2|ds| = shear_px pixels along
 *               shear_angle, bias theta; transfer P(k) 2i sin(k.ds + theta)
 *   bevel_slope prism chamfer slope s_b; chord = clamp(2 s_b d, 0, T) with d
 *               the in-plane distance to the nearest side wall (um)
 */
typedef struct {
    int32_t H, W;
    double dx_um, lambda_um, NA, n_medium, defocus_um;
    uint32_t modes;
    double oblique_frac, oblique_angle;
    double shear_px, shear_angle, bias_phase;
    double bevel_slope;
} osog_optics_t;

/*
 * Tuning of the batched path (osog_batch_submit).  Zero fields take the
 * value osog_autotune stored in the plan for this batch shape, else the
 * default.
 *   pairs_per_particle  particle-band pairs reserved per particle (default: the
 *                       plan's, see osog_plan_set_pairs_per_particle)
 *   use_graph           1: replay the launch sequence as a CUDA graph that the
 *                       plan caches per batch shape; 0 (or -1): launch directly
 *   persistent          1: the three render stages of each group of up to 32
 *                       scenes run as one persistent launch that pulls work
 *                       items from a device queue (square canvases only);
 *                       -1: three launches (default)
 *   band_rows           rows per binning band (the raster's tile height): a
 *                       multiple of the strip height R that divides H and
 *                       gives at most 64 bands (R = 8192 / W rows for
 *                       W >= 1024, 4 for 128 <= W <= 512, 512 / W below);
 *                       0 = the default max(H / 64, 16, R)
 *   wait_polls          polls before a bounded device wait gives up and
 *                       latches OSOG_ERR_TIMEOUT: in the persistent launch the
 *                       wait for another stage's work (about 0.1 us apart,
 *                       0 = 2^24; after one wait has given up the launch's
 *                       later waits return at once), in the column pass of a
 *                       square canvas of 1024 or more the wait for the bulk
 *                       copy of its column block (0 = 2^20); the launch always
 *                       ends
 *   test_wait_extra     failure-detection test (0 = off): raises the number of
 *                       finished strips each column item of the persistent
 *                       launch waits for by this many, and makes the column
 *                       pass's bulk-copy barrier expect 16 bytes more than its
 *                       copy delivers, so those waits run out; the images of
 *                       such a launch are invalid
 *   raster              1: rasterise in a kernel of its own over tiles of one
 *                       band by a few hundred columns, handing the per-pixel
 *                       phase and absorption words to the strip pass through
 *                       the filtered-spectrum region; -1: inside the strip
 *                       pass (default).  Both give bitwise the same images.
 */
typedef struct {
    int32_t pairs_per_particle;
    int32_t use_graph;
    int32_t persistent;
    int32_t band_rows;
    int32_t wait_polls;
    int32_t test_wait_extra;
    int32_t raster;
    int32_t reserved;
} osog_tuning_t;

/*
 * Create a plan for H x W canvases: uploads FP64-built twiddle tables
 * exp(-2 pi i k / N) rounded to float32 and allocates the device status
 * word.  Returns OSOG_ERR_UNSUPPORTED_SIZE for a bad size, OSOG_ERR_CUDA if
 * the device allocation fails.  *plan is NULL on failure.
 */
int osog_plan_create(osog_plan_t **plan, int32_t H, int32_t W);

/* Release a plan and its device memory (NULL is ignored).  The caller must
 * make sure no work using the plan is still running. */
void osog_plan_destroy(osog_plan_t *plan);

/*
 * Workspace bytes needed by a render of `batch` scenes holding `n_max`
 * particles in total with K modalities (osog_render: batch = 1).  The
 * workspace is a caller-owned device buffer aligned to 256 bytes.  Returns
 * 0 for invalid arguments.
 */
size_t osog_workspace_size(const osog_plan_t *plan, int32_t n_max, int32_t K,
                           int32_t batch);

/*
 * Forward render of one scene (the whole path, Sec. III.A-C).
 *   soa      device float32 [9][ld], n particles in columns 0..n-1
 *   n        particle count, 0 <= n <= ld (0 renders an empty field)
 *   optics   host struct; optics->H, ->W must equal the plan's size
 *   image    device float32 [K][H][W], written completely
 *   ws       device workspace of ws_bytes >= osog_workspace_size(plan, n, K, 1)
 * Returns OSOG_OK or a host-side error; device-side errors are latched.
 */
int osog_render(osog_plan_t *plan, const float *soa, int64_t ld, int32_t n,
                const osog_optics_t *optics, float *image, void *ws,
                size_t ws_bytes, osog_stream_t stream);

/*
 * Forward render of one scene that may hold general convex polyhedra
 * (kind 2): each is the intersection of its own half-spaces
 * a_x u + a_y v + a_z z <= b (Eq. 1 with the caller's M planes), u, v in um
 * in the particle's frame (centre cx, cy; rotated by theta), z in um along
 * the optical axis; its thickness is the vertical chord through the pixel
 * centre.  Kinds 0 and 1 render as in osog_render.
 *   planes         device float32 [n_planes][4] rows (a_x, a_y, a_z, b),
 *                  16-byte aligned
 *   plane_offsets  device int32 [n + 1]: particle p owns rows
 *                  plane_offsets[p] .. plane_offsets[p+1]-1 (1..32 of them
 *                  for kind 2; ignored for kinds 0 and 1)
 *   soa rows 3 and 4 of a kind-2 particle hold the circumscribed radius of
 *   its footprint in px (both > 0); T is not used.
 *   ws             >= osog_polyhedra_workspace_size(plan, n, K, n_planes)
 * A kind-2 particle with a bad plane range latches
 * OSOG_ERR_INVALID_PARTICLE, non-finite planes OSOG_ERR_NONFINITE_INPUT,
 * and is skipped.  Other arguments and errors as for osog_render.  The
 * adjoint (osog_render_backward) covers kinds 0 and 1 only.
 */
size_t osog_polyhedra_workspace_size(const osog_plan_t *plan, int32_t n_max, int32_t K,
                                     int32_t n_planes);
int osog_render_polyhedra(osog_plan_t *plan, const float *soa, int64_t ld, int32_t n,
                          const float *planes, const int32_t *plane_offsets,
                          int32_t n_planes, const osog_optics_t *optics, float *image,
                          void *ws, size_t ws_bytes, osog_stream_t stream);

/*
 * DIC image of one scene in the literal (incoherent) reading of Eq. 5: the
 * exit wave U itself is sheared by +-ds (ds = shear_px / 2 pixels along
 * shear_angle) and interfered at bias theta,
 *   J = |U(r + ds) e^{i theta} - U(r - ds) e^{-i theta}|^2,
 * and J is convolved with the intensity point spread function |h|^2 of the
 * brightfield pupil (NA, defocus; h = IDFT2(P)), normalised to unit sum:
 *   image = J (*) |h|^2 / sum |h|^2   (device float32 [H][W]).
 * optics->modes is ignored; oblique settings are not used.  Workspace:
 * osog_dic_incoherent_workspace_size(plan, n).  Errors as for osog_render.
 * (osog_render's DIC modality is the coherent reading: the sheared
 * difference taken through the pupil.)
 */
size_t osog_dic_incoherent_workspace_size(const osog_plan_t *plan, int32_t n_max);
int osog_render_dic_incoherent(osog_plan_t *plan, const float *soa, int64_t ld, int32_t n,
                               const osog_optics_t *optics, float *image, void *ws,
                               size_t ws_bytes, osog_stream_t stream);

/*
 * Sensor noise (Sec. III.C: Poisson photon shot noise plus Gaussian read
 * noise, N ~ P(lambda) + G(0, sigma^2)) applied to `count` intensities:
 *   out[i] = (Poisson(g max(image[i], 0)) + read_sigma Z_i) / g,
 * g = photons_per_unit (photo-electrons per unit intensity, 0 < g <= 1e12),
 * read_sigma >= 0 in electrons, Z_i standard normal; the noiseless mean is
 * the input.  Random numbers: Philox4x32-10 keyed by `seed`, counter (i,
 * round, tag), so each element's draw depends only on (seed, i) and not on
 * the launch; Poisson by inversion below rate 10 and by transformed
 * rejection (PTRS) above, decided in double precision.  image and out are
 * device float32 arrays (may be the same).  Returns OSOG_ERR_INVALID_ARG for
 * bad arguments.
 */
int osog_sensor_noise(const float *image, int64_t count, double photons_per_unit,
                      double read_sigma, uint64_t seed, float *out, osog_stream_t stream);

/*
 * Stage entry: rasterise only.  Writes the OPD and ATT maps of Eq. 2 as a
 * device float32 [H][W][2] array (opd, att per pixel), in the same order of
 * summation as osog_render.  Workspace as for osog_render with K = 1.
 */
int osog_render_opd(osog_plan_t *plan, const float *soa, int64_t ld, int32_t n,
                    const osog_optics_t *optics, float *opd_att, void *ws,
                    size_t ws_bytes, osog_stream_t stream);

/*
 * Stage entry: optics only.  Takes a device float32 [H][W][2] OPD/ATT map,
 * forms the exit wave (Eq. 2, Eq. 4) and images every selected modality
 * into device float32 [K][H][W].  Workspace: osog_workspace_size(plan, 0, K, 1).
 */
int osog_optics_from_opd(osog_plan_t *plan, const float *opd_att,
                         const osog_optics_t *optics, float *image, void *ws,
                         size_t ws_bytes, osog_stream_t stream);

/*
 * Workspace bytes needed by osog_render_backward for n_max particles and K
 * modalities (0 for invalid arguments).
 */
size_t osog_backward_workspace_size(const osog_plan_t *plan, int32_t n_max, int32_t K);

/*
 * Gradient of a loss of the images of one scene (the adjoint of
 * osog_render; the paper's end-to-end differentiability, Sec. III.C and
 * Sec. IV.B).  Given grad_image = dL/dI (device float32 [K][H][W]) it writes
 *   grad_soa     device float32 [9][ld]: dL/d(cx, cy, theta, a|hx, b|hy, T,
 *                dn, mu) of particles 0..n-1 in the units of the particle
 *                tensor; the kind row and particles skipped as invalid get 0
 *   grad_optics  device float32 [4]: dL/d(defocus_um, shear_px, shear_angle,
 *                bias_phase); the shear and bias entries are zero unless the
 *                DIC modality is selected
 * The forward intermediates are recomputed, not read from an earlier render
 * (osog_render_keep + osog_render_backward_kept below keep them instead);
 * every sum runs in a fixed order (bitwise reproducible).  The pupil circle
 * is a hard cut-off, so NA has no gradient.  Workspace:
 * osog_backward_workspace_size(plan, n, K).  Errors as for osog_render.
 */
int osog_render_backward(osog_plan_t *plan, const float *soa, int64_t ld, int32_t n,
                         const osog_optics_t *optics, const float *grad_image,
                         float *grad_soa, float *grad_optics, void *ws, size_t ws_bytes,
                         osog_stream_t stream);

/*
 * The forward render and its adjoint with the forward intermediates kept
 * between the two calls instead of recomputed (the usual way a training or
 * inverse-rendering step runs: one forward, then one backward).
 *
 * osog_render_keep writes the images exactly as osog_render does (same
 * arguments, same results) and leaves the particle records, band bins and
 * filtered spectra of the scene in ws, which must hold
 * osog_backward_workspace_size(plan, n, K) bytes.
 *
 * osog_render_backward_kept then computes what osog_render_backward computes
 * (same arguments, same results) from that state.  It accepts only the ws
 * pointer and size, soa pointer, ld, n and optics (compared field by field)
 * of an earlier osog_render_keep on this plan, and fails with
 * OSOG_ERR_INVALID_ARG otherwise.  Any other call of this plan that writes
 * the same ws drops the state, and the adjoint consumes it: a second
 * backward needs a new osog_render_keep (or osog_render_backward, which
 * recomputes).  The caller keeps the particle values and ws untouched
 * between the two calls; a changed particle tensor at the same address is
 * not detected.  The plan remembers the states of its last 64 workspaces.  Errors
 * otherwise as for osog_render and osog_render_backward.
 */
int osog_render_keep(osog_plan_t *plan, const float *soa, int64_t ld, int32_t n,
                     const osog_optics_t *optics, float *image, void *ws, size_t ws_bytes,
                     osog_stream_t stream);
int osog_render_backward_kept(osog_plan_t *plan, const float *soa, int64_t ld, int32_t n,
                              const osog_optics_t *optics, const float *grad_image,
                              float *grad_soa, float *grad_optics, void *ws, size_t ws_bytes,
                              osog_stream_t stream);

/*
 * Bind a device array of the four differentiable optics scalars to the plan:
 *   params_dev  device float32 [4]: defocus_um, shear_px, shear_angle,
 *               bias_phase (the order of grad_optics)
 * While bound, every render and adjoint of this plan (all entry points that
 * take a plan) reads these four values on the device when its kernels run,
 * and ignores the optics struct's own four fields; the struct's other fields
 * apply as before.  A CUDA graph captured from such calls therefore sees the
 * values a device-side update writes between replays (an inverse-rendering
 * step without a device-to-host read of the optics).  The array stays the
 * caller's and must outlive the binding and any graph that uses it; its
 * values are not checked (non-finite values give non-finite images).  NULL
 * unbinds.  OSOG_ERR_INVALID_ARG for a NULL plan or a pointer that is not
 * 4-byte aligned.
 */
int osog_plan_bind_optics_params(osog_plan_t *plan, const float *params_dev);

/*
 * Particle-band pairs reserved per particle (default 8) by this plan's
 * single-scene calls (osog_render, osog_render_opd, osog_render_keep, the
 * adjoint, the polyhedra and incoherent-DIC renders), by the batched path
 * when its tuning leaves pairs_per_particle at 0, and by every workspace-size
 * query of the plan; query the workspace size after setting it.  A particle
 * whose bounding rectangle meets more bands than reserved latches
 * OSOG_ERR_BIN_OVERFLOW.  Drops the plan's kept forward states.
 * OSOG_ERR_INVALID_ARG unless 1 <= pairs_per_particle <= 64.
 */
int osog_plan_set_pairs_per_particle(osog_plan_t *plan, int32_t pairs_per_particle);

/*
 * The reservation that a scene needs when no particle's bounding rectangle
 * reaches further than max_half_extent_px from its centre along y (a + b is
 * a bound for every kind: the half-height of an ellipse or of a rotated
 * rectangle with half-lengths a, b, and the radius a of a polyhedron),
 * given the plan's band height; 0 for a negative or non-finite extent.
 */
int32_t osog_pairs_for_extent(const osog_plan_t *plan, double max_half_extent_px);

/*
 * Batched forward render of S scenes that share the plan's H x W and the/*
 * Batched forward render of S scenes that share the plan's H x W and the
 * same modality bits (per-scene optics may otherwise differ).
 *   soa_all  device float32 [9][ld]; scene s owns columns
 *            offsets[s] .. offsets[s+1]-1
 *   offsets  HOST int32 [S+1], non-decreasing, offsets[S] <= ld
 *   optics   HOST array of S structs
 *   images   device float32 [S][K][H][W]
 *   tuning   NULL for defaults
 *   ws       >= osog_workspace_size(plan, offsets[S]-offsets[0], K, S)
 */
int osog_batch_submit(osog_plan_t *plan, const float *soa_all, int64_t ld,
                      const int32_t *offsets, int32_t S,
                      const osog_optics_t *optics, float *images,
                      const osog_tuning_t *tuning, void *ws, size_t ws_bytes,
                      osog_stream_t stream);

/*
 * Autotuner of the batched path.  For this batch shape it measures, for
 * each candidate band height (the smallest valid one and up to three
 * doublings), the exact particle-band pairs per particle the batch needs (a
 * binning dry run), then times the batch five times with three launches
 * per group (the raster inside the strip pass, and in a tile kernel of its
 * own) and, on square canvases, with the persistent launch, and keeps the
 * candidate with the fastest median.  The choice is stored in the plan for (S, total particles,
 * K) and used by later osog_batch_submit calls of that shape whose tuning
 * leaves the fields at 0; it is also written to *out when out is not NULL.
 * Arguments as for osog_batch_submit; images receive a valid render.  This
 * call synchronises the stream and must not be captured into a graph.
 */
int osog_autotune(osog_plan_t *plan, const float *soa_all, int64_t ld,
                  const int32_t *offsets, int32_t S, const osog_optics_t *optics,
                  float *images, void *ws, size_t ws_bytes, osog_stream_t stream,
                  osog_tuning_t *out);

/*
 * Image losses of inverse rendering (Sec. IV.B), evaluated with the
 * library's FFT passes: K float32 images of the plan's H x W against K
 * target images, with A_k and B_k their unnormalised forward 2-D DFTs.
 *   misfit     the coarse-to-fine curriculum's low-pass misfit,
 *              misfit_scale sum_k sum_px (lp(I_k) - lp(T_k))^2 with lp the
 *              ideal low-pass filter |f| <= cutoff (cycles/um, on the grid
 *              fftfreq(W, dx_um) x fftfreq(H, dx_um)), computed by Parseval
 *              as misfit_scale / (H W) sum_{|f| <= cutoff} |A - B|^2;
 *   spectral   Eq. 8, the squared difference of the log-amplitude spectra,
 *              1 / (K H W) sum_k sum_f (log(|A_k| + e_k) - log(|B_k| + e_k))^2
 *              with the guard e_k = eps_rel max_f |B_k(f)| (the paper writes
 *              log|F(.)|; the guard keeps frequencies where both spectra are
 *              rounding noise from dominating; float32 spectra carry noise of
 *              ~1e-7 of their largest amplitude, so eps_rel >= 1e-5).
 *
 * osog_loss_target stores the targets' spectra and largest amplitudes in a
 * caller-owned device table of osog_loss_table_size(plan, K) bytes (256-byte
 * aligned); one table serves any number of osog_image_loss calls.
 *   target  device float32 [K][H][W], 1 <= K <= 32
 *
 * osog_image_loss writes, on the device,
 *   loss[0] = misfit (0 when misfit_scale is 0), loss[1] = spectral loss
 *   (0 when spectral_weight is 0), and, when grad_image is not NULL,
 *   grad_image = d(misfit + spectral_weight spectral)/dI (float32 [K][H][W]).
 * The cutoff is read from device memory when the kernels run, so a CUDA
 * graph captured from this call follows a cutoff updated on the device.
 * Every sum runs in a fixed order (bitwise reproducible).  Both calls take a
 * workspace of osog_loss_workspace_size(plan, K) bytes.  Host-side errors:
 * OSOG_ERR_INVALID_ARG (bad K, pointer or parameter), OSOG_ERR_WORKSPACE.
 */
typedef struct {
    double dx_um;            /* pixel pitch (the misfit's frequency grid) */
    const float *cutoff;     /* device float: low-pass radius (cycles/um); needed when
                                misfit_scale != 0 */
    double misfit_scale;     /* 0: no misfit */
    double spectral_weight;  /* weight of Eq. 8 in the gradient; 0: not evaluated */
    double eps_rel;          /* > 0: guard of the logarithms */
} osog_loss_t;

size_t osog_loss_table_size(const osog_plan_t *plan, int32_t K);
size_t osog_loss_workspace_size(const osog_plan_t *plan, int32_t K);
int osog_loss_target(osog_plan_t *plan, const float *target, int32_t K, void *table,
                     size_t table_bytes, void *ws, size_t ws_bytes, osog_stream_t stream);
int osog_image_loss(osog_plan_t *plan, const float *image, int32_t K, const void *table,
                    size_t table_bytes, const osog_loss_t *params, float *loss,
                    float *grad_image, void *ws, size_t ws_bytes, osog_stream_t stream);

/* Synchronise `stream`, return the first device-latched status since the
 * last call (OSOG_OK if none) and clear it. */
int osog_sync_status(osog_plan_t *plan, osog_stream_t stream);

/* Text of the last host-side error of the calling thread ("" if none). */
const char *osog_last_error(void);

/* Number of kernels this plan has launched since it was created (graph
 * replays count each kernel node once per replay). */
int64_t osog_plan_launch_count(const osog_plan_t *plan);

/*
 * Per-kernel timing.  Between osog_profile_begin and osog_profile_end every
 * kernel the plan launches is bracketed by CUDA events on its stream (graph
 * replay is disabled meanwhile).  osog_profile_end synchronises `stream`
 * and writes, per kernel class (OSOG_KERNEL_*), the summed device time in
 * milliseconds and the launch count.  Arrays have OSOG_KERNEL_CLASS_COUNT
 * entries.  At most 8192 launches are timed per session; later ones are
 * counted but not timed.  A single scene of at most 256 particles is binned
 * by one launch (count, scan and fill together), counted as
 * OSOG_KERNEL_BIN_COUNT.
 */
int osog_profile_begin(osog_plan_t *plan);
int osog_profile_end(osog_plan_t *plan, osog_stream_t stream, float *ms,
                     int32_t *launches);

/*
 * Forward render that allocates nothing (no counterpart in the paper).
 * For callers that cannot call cudaMalloc, or cannot create a plan, because
 * their host application owns all device memory (a plugin inside another
 * framework, a real-time loop that may not block on an allocator).  Same
 * arguments and result as osog_render minus the plan and the workspace: the
 * twiddle tables, the status word and every intermediate buffer live in
 * static device arrays of the library (8 MiB of scratch plus 33 KB of
 * tables) that each GPU loading the library keeps until the process exits.
 *   Limit: the render's scratch must fit in 8 MiB, e.g. a 256 x 256 canvas
 *   with 3 modalities and up to ~50,000 particles, or 512 x 512 with one
 *   modality and up to ~33,000; larger renders return OSOG_ERR_WORKSPACE
 *   before any device work.  The particle-band lists get the scratch that the
 *   other regions leave (at least one slot per particle); a scene whose
 *   particles span more bands than that latches OSOG_ERR_BIN_OVERFLOW and
 *   renders without the pairs that did not fit.  Other host-side errors:
 *   OSOG_ERR_INVALID_ARG, OSOG_ERR_UNSUPPORTED_SIZE, OSOG_ERR_CUDA;
 *   osog_last_error is not set.
 *   The first call on a device sets that device up (resolves the static
 *   arrays' addresses, uploads the tables, sets kernel attributes); make it
 *   before any stream capture.
 *   All calls share the static scratch: calls that overlap on the GPU (on
 *   different streams, or from different threads) race and must be ordered
 *   by the caller.  Device-side errors (invalid or non-finite particles,
 *   bin overflow) latch in one status word per device, shared by every call
 *   of this entry point and kept until osog_noalloc_sync_status reads it.
 */
int osog_render_noalloc(const float *soa, int64_t ld, int32_t n,
                        const osog_optics_t *optics, float *image,
                        osog_stream_t stream);

/*
 * Status of osog_render_noalloc on the current device (allocates nothing):
 * synchronises `stream`, returns the first code latched by any
 * osog_render_noalloc call on this device since the last read (OSOG_OK if
 * none) and clears it.  OSOG_ERR_CUDA if a runtime call fails.
 */
int osog_noalloc_sync_status(osog_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* OSOG_H */
