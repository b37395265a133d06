/* gr.h -- C ABI of the GB300 generalized-ray path tracer (libgr.so).
 *
 * Backward (sensor-to-source) Monte Carlo transport of generalized rays,
 * "A Generalized Ray Formulation For Wave-Optics Rendering" (Steinberg et al.,
 * arXiv 2303.15762):
 *   - a pixel sources generalized rays {r0, k0, beta, rho = 0}      (Sec. 4.1, Eq. MC_sourcing;
 *     detector as coherent states, Sec. 3.2, Eq. wdf_coherent_states)
 *   - rays propagate by ray tracing, their footprint per Eq. K_free_space_propagation
 *     (interactive simplification, Sec. 7.2)
 *   - at a surface the interaction acts on the wavevector-reversed ray  (Eq. action_time_reversal)
 *     and one child ray is sampled                                      (Eq. MC_light_transport_Q1):
 *     grating orders (Eq. K_grating), rough-surface lobe (Eq. K_surface_HS),
 *     smooth reflection with a Fresnel Mueller weight (Eq. K_reflection_refraction)
 *   - light sources are integrated by the measurement operator          (Eq. measurement_operator)
 *   - the per-pixel intensity is the sample mean                        (Algorithm 1)
 * The output is the intensity per detector element: per view, pixel, spectral
 * bin and Stokes component.
 *
 * Conventions (all calls):
 *   - every call returns gr_status; out-pointers are written only on GR_OK;
 *     gr_last_error() gives a thread-local message for the last failure;
 *     no C++ exception crosses this boundary.
 *   - host pointers are read during the call only (the caller keeps ownership);
 *     device pointers passed in are borrowed until the work enqueued on the
 *     given stream completes.
 *   - stream arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream); work is enqueued asynchronously and the caller
 *     synchronises on its own stream.
 *   - units: scene geometry in metres; optical lengths (wavelengths, grating
 *     period and height, roughness, correlation and coherence lengths, pixel
 *     pitch) in micrometres.
 */
#ifndef GR_H
#define GR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GR_OK = 0,
  GR_E_INVALID = 1, /* bad argument or descriptor */
  GR_E_OOM = 2,     /* device allocation failed */
  GR_E_CUDA = 3,    /* a CUDA runtime call failed */
  GR_E_TIMEOUT = 4, /* the render loop exceeded its iteration limit */
  GR_E_BUSY = 5     /* object in use */
} gr_status;

typedef struct gr_scene gr_scene;
typedef struct gr_frame gr_frame;

/* Material kinds (interaction operators, Sec. 6). */
enum {
  GR_MAT_ABSORBER = 0, /* black: terminates paths */
  GR_MAT_GRATING = 1,  /* sinusoidal grating, Eq. K_grating */
  GR_MAT_ROUGH = 2,    /* Gaussian-statistics rough surface, Eq. K_surface_HS */
  GR_MAT_MIRROR = 3,   /* smooth reflector, Eq. K_reflection_refraction */
  GR_MAT_EMITTER = 4,  /* emissive geometry light source (Sec. 7.2) */
  GR_MAT_DIELECTRIC = 5 /* smooth refracting interface, Eq. K_reflection_refraction */
};

/* One material, 64 bytes.  fresnel: 0 = unit reflectance (Mueller identity),
 * 1 = conductor with complex index n_re + i n_im (Fresnel Mueller matrix at the
 * incidence angle, also scaling diffractive lobes).
 * Grating: period_um (Lambda), height_um (h, peak to peak; order weights
 * J_j(h k / 2)^2), gdir = grating vector direction in world space (projected
 * onto the surface tangent plane at the hit).
 * Rough: sigma_h_um (RMS height), corr_len_um (Gaussian correlation length).
 * Emitter: Le (exitance), coh_len_um (coherence length; angular spread
 * lambda / coh_len per axis, Eq. coherence_diffusivity; 0 = coherent).  An
 * emitter is the planar set of triangles carrying the same emitter material;
 * only its front face (counter-clockwise winding) emits.
 * Dielectric: refractive index n(lambda) = n_re + cauchy_b_um2 / lambda^2
 * (lambda in um); the front face (counter-clockwise winding) looks out into
 * air (index 1), so a dielectric body is a closed mesh wound outward; media do
 * not nest.  Reflection or refraction is chosen by the Fresnel reflectance
 * (Mueller weights in s-p frames, total internal reflection past the critical
 * angle); inside, the footprint propagates with |k| = n k0. */
typedef struct {
  int32_t type;
  int32_t fresnel;
  float n_re, n_im;
  float period_um, height_um;
  float gdir[3];
  float sigma_h_um, corr_len_um;
  float Le, coh_len_um;
  float cauchy_b_um2;
  float reserved[2];
} gr_material;

/* Light sources measured on escape (Sec. 7.2): distant source of irradiance E
 * toward unit direction dir with coherence length coh_len_um (0 = spatially
 * coherent), or a constant environment of radiance E (dir ignored). 32 bytes. */
enum { GR_LIGHT_DISTANT = 0, GR_LIGHT_ENV = 1 };
typedef struct {
  int32_t type;
  float dir[3];
  float E;
  float coh_len_um;
  float reserved[2];
} gr_light;

/* Scene description (host memory, read during gr_scene_create only).
 * verts: float32 [n_tris][3][3] (three vertices, xyz); tri_mat: int32 [n_tris]
 * material index per triangle.  n_tris may be 0 (every ray escapes). */
typedef struct {
  int32_t n_tris;
  const float* verts;
  const int32_t* tri_mat;
  int32_t n_mats;
  const gr_material* mats;
  int32_t n_lights;
  const gr_light* lights;
} gr_scene_desc;

/* A detector (Sec. 3.2 detector distribution D): a pinhole camera (or an
 * orthographic one, ortho = 1) of width x height pixels, each sourcing
 * generalized rays with beta = f_beta * p_pix_um, rho = 0, alpha = 1 and one
 * wavelength per path from n_bins bins spanning [lambda_min_um, lambda_max_um]
 * (bin b = sample mod n_bins).  n_stokes is 1 (unpolarised intensity) or 4
 * (Stokes vector in the camera's right/up frame).  max_depth counts surface
 * interactions.  A render adds the samples [first_sample, first_sample + spp)
 * of every pixel.  view_index keys the random stream; scene_index selects the
 * scene in gr_render's scene list.  100 bytes. */
typedef struct {
  float eye[3], look_at[3], up[3];
  float vfov_deg;
  int32_t width, height;
  float p_pix_um, f_beta;
  float lambda_min_um, lambda_max_um;
  int32_t n_bins, n_stokes, max_depth;
  int32_t spp, first_sample;
  int32_t view_index, scene_index;
  int32_t ortho;
  float ortho_half_m;
} gr_view_desc;

/* Render options (36 bytes).  flags: GR_FLAG_NEE next-event estimation toward emitters
 * with power-heuristic MIS; GR_FLAG_RR Russian roulette after 3 interactions;
 * GR_FLAG_NO_RENORM keeps raw grating order weights (no renormalisation over
 * propagating orders); the default tree is the binary BVH with its child
 * boxes stored in FP16, rounded outward (32 bytes per node; used when every
 * coordinate of every scene of the call is within +-16384); GR_FLAG_FP32_NODES
 * walks the same tree with FP32 child boxes (64 bytes per node);
 * GR_FLAG_WIDE_BVH traverses the 4-wide BVH with 8-bit quantised child boxes
 * (all three give the same closest hits: a box that contains the FP32 box is
 * entered whenever the FP32 box is; the wide tree halves node visits but needs
 * more registers per thread); GR_FLAG_HERO hero-wavelength spectral MIS (Sec. 7.2):
 * with n_bins a multiple of 4, a path's bin is the hero of the class of bins
 * {c, c+Q, c+2Q, c+3Q} (Q = n_bins/4) and drives every sampling decision;
 * every connection to a light (escape, emitter hit, next-event estimate) is
 * measured at all four wavelengths, each with its own footprint, and weighted
 * by multiple importance sampling over the class wavelengths' path densities
 * (zero for a wavelength after a dispersive delta: a grating order j != 0 or
 * a dispersive dielectric) -- the balance heuristic where only lobe sampling
 * could make the path, the power heuristic over (wavelength, lobe or emitter
 * sampling) where next-event estimation could too; each bin is still divided
 * by the number of samples whose hero it is (GR_E_INVALID if n_bins % 4 != 0; not available in
 * gr_render_static); GR_FLAG_ANISO anisotropic footprints (Sec. 3.1: beta and rho as
 * matrices): each ray carries the complex 2x2 K = A^-1 of its transverse field
 * exp(-x^T A x / 2), propagates it exactly (K + i z/|k| I), maps it through every
 * interaction by the surface's anamorphic projection (orthogonal for mirrors; the
 * grating and Snell anamorphic factors for orders and refraction) and measures sources
 * with its anisotropic wavevector and footprint Gaussians; a path that meets only
 * mirror reflections renders as without the flag (not combined with GR_FLAG_HERO;
 * not available in gr_render_static).  table_dtype: storage of the grating order tables
 * (GR_TABLE_F32 / F16 / BF16); arithmetic is FP32 either way.  pool_size:
 * wavefront slots, i.e. path samples in flight (0 = one slot per ticket -- a
 * ticket is one pixel's samples of one wavelength bin, or with GR_FLAG_HERO
 * one of min(4, spp / Q) consecutive ranges (1 if spp < 2 Q) of one pixel's
 * samples of one class of 4 bins (Q = n_bins / 4; split ranges' sums meet in
 * a 260-byte record per class and pixel and are added in range order) --
 * capped at 2^25 slots and at a quarter of the device memory free at the
 * call; at most 2^30 - 256; a slot takes 265 bytes,
 * plus 164 with GR_FLAG_HERO and 80 with GR_FLAG_ANISO; images do not depend on it);
 * block: threads per block (0 = default). */
enum { GR_FLAG_NEE = 1, GR_FLAG_RR = 2, GR_FLAG_NO_RENORM = 4, GR_FLAG_WIDE_BVH = 8, GR_FLAG_HERO = 16, GR_FLAG_ANISO = 32,
       GR_FLAG_FP32_NODES = 64 };
enum { GR_TABLE_F32 = 0, GR_TABLE_F16 = 1, GR_TABLE_BF16 = 2 };
typedef struct {
  uint32_t seed;
  int32_t flags;
  int32_t table_dtype;
  int32_t pool_size;
  int32_t block;
  int32_t use_graph;     /* 1: run the whole render as ONE graph launch: a CUDA graph
                             whose conditional while-node repeats the wavefront iteration
                             until every ticket is done (device-side loop, bounded by the
                             iteration limit); the instantiated graph is cached in the
                             frame and reused while the launch shapes are unchanged; the
                             call waits for completion */
  int32_t max_iterations; /* 0 = default bound; exceeding it returns GR_E_TIMEOUT */
  int32_t profile;        /* 1: time every kernel with CUDA events on the render stream
                             (not with use_graph); the call then waits for completion */
  int32_t regen_threshold_pct; /* 0: refill idle slots every iteration; p > 0: claim new
                                  tickets only once at least p% of the pool is idle (fresh
                                  camera rays then enter in coherent groups) */
} gr_render_opts;

/* Render statistics of the last gr_render on a frame (device-side counters,
 * read after the stream is synchronised). */
typedef struct {
  int64_t samples;        /* path samples completed */
  int64_t segments;       /* ray segments traced (camera + continuation) */
  int64_t shadow_rays;    /* NEE shadow rays traced (directions that cannot reach their emitter are not requested) */
  int64_t refine64_hits;  /* ray-triangle tests decided in FP64 */
  int64_t refine64_lobes; /* grating / Poisson choices decided in FP64 */
  int64_t iterations;     /* wavefront iterations */
  int64_t kernel_launches;
  int64_t node_visits;    /* BVH internal nodes visited (trace + shadow) */
  int64_t tri_tests;      /* ray-triangle tests (trace + shadow) */
  /* last render with profile = 1: device ms and launches per kernel
     (0 regen, 1 trace: the trace queue and the next-event rays, 2 shade,
     3 shadow: the next-event measurement) */
  double kernel_ms[4];
  int64_t kernel_count[4];
} gr_stats;

/* Upload a scene: the interaction operators of Sec. 6 (per-triangle
 * materials: grating Eq. K_grating, rough surface Eq. K_surface_HS, smooth
 * reflection and refraction Eq. K_reflection_refraction) and the sourcing
 * distributions the measurement operator integrates (Eq. measurement_operator:
 * distant sources and emissive triangle sets, Sec. 7.2).  The geometry is
 * traced as rays (Sec. 7.2: footprints are small against geometric detail), so
 * a BVH is built on the device: 30-bit Morton order, then agglomerative
 * clustering along that order (PLOC, window +-8, least merged surface area);
 * topology and FP32 bounds are deterministic.  The binary tree is also
 * collapsed into a 4-wide BVH with 8-bit quantised, conservatively rounded
 * child boxes.  desc arrays are host memory, read during the call only; the
 * library owns the device copy until gr_scene_destroy.  The scene belongs to
 * the device current at creation and may only be rendered there.
 * Errors: GR_E_INVALID (null/negative sizes, material index out of range,
 * unknown material or light type), GR_E_OOM, GR_E_CUDA. */
gr_status gr_scene_create(const gr_scene_desc* desc, void* cuda_stream, gr_scene** out);
gr_status gr_scene_destroy(gr_scene* scene);
/* Device bytes the scene holds (triangles, BVH layouts, materials, lights,
 * emitters); host-side bookkeeping, no CUDA call.  Errors: GR_E_INVALID. */
gr_status gr_scene_bytes(const gr_scene* scene, size_t* bytes_out);

/* Frame = the detector elements' accumulators for n_views views.  A view is
 * a detector (Sec. 3.2, Eq. wdf_coherent_states: each pixel a set of coherent
 * states), and its output is the intensity per detector element (Algorithm 1:
 * the mean over the element's samples), resolved per spectral bin and Stokes
 * component.  For each view the frame holds a float32 sum and a Kahan
 * compensation per [bin][y][x][stokes], plus per-bin sample counts (host
 * side).  gr_frame_create allocates them on the device (library-owned,
 * zero-initialised on stream).  The frame belongs to the current device.
 * Errors: GR_E_INVALID, GR_E_OOM, GR_E_CUDA. */
gr_status gr_frame_create(const gr_view_desc* views, int32_t n_views, void* cuda_stream, gr_frame** out);

/* A frame over caller-owned accumulators (e.g. a torch tensor).
 * accum_device: device memory of the current device holding 2 * T float32,
 * T = the sum over views of width * height * n_bins * n_stokes: the per-view
 * sums laid out view after view as [bin][y][x][stokes], then their Kahan
 * compensations in the same order (the layout gr_render_static uses).  The
 * buffer is borrowed until gr_frame_release; it is not cleared, renders add
 * into it, and gr_readback's means assume it held zeros at wrap time (the
 * frame's sample counts start at zero).  gr_frame_reset zeroes it.  The mean of
 * an element is (sum - compensation) / count.  accum_device == NULL is
 * gr_frame_create (library-owned accumulators).  Host or other-device pointers
 * are rejected with GR_E_INVALID (the buffer's size cannot be checked: it
 * must hold 2 * T floats).  Errors: GR_E_INVALID, GR_E_OOM, GR_E_CUDA. */
gr_status gr_frame_wrap(const gr_view_desc* views, int32_t n_views, float* accum_device, void* cuda_stream,
                        gr_frame** out);
/* Device bytes the frame holds now: its library-owned accumulators (none for
 * a wrapped buffer), its counters and the wavefront scratch kept from its last
 * render (a render grows it to gr_render_scratch_bytes when it is smaller).
 * Host-side bookkeeping, no CUDA call.  Errors: GR_E_INVALID. */
gr_status gr_frame_bytes(const gr_frame* frame, size_t* bytes_out);
/* Zero the frame's accumulators (on stream) and its sample counts. */
gr_status gr_frame_reset(gr_frame* frame, void* cuda_stream);
/* Free the frame (library-owned accumulators included; a wrapped buffer stays
 * the caller's).  Synchronises the device. */
gr_status gr_frame_release(gr_frame* frame);

/* Enqueue the samples [first_sample, first_sample + spp) of every view on the
 * stream, adding them into frame (which must have been created for views of
 * the same shapes).  Each sample is one path of Algorithm 1: a generalized
 * ray sourced from the pixel (Eq. MC_sourcing; Sec. 7.2: uniform position on
 * the pixel, rho = 0, beta = f_beta * p_pix_um, one wavelength bin), traced
 * through scenes[view.scene_index] with the footprint update of
 * Eq. K_free_space_propagation, interacting by sampling one child ray per
 * vertex (Eq. MC_light_transport_Q1) and measured against the sources
 * (Eq. measurement_operator).  Accumulation is per pixel and bin in sample
 * order (deterministic).  Scenes and frame must belong to the current device.
 * Errors: GR_E_INVALID (shape mismatch, bad scene index, bad options, scene or
 * frame of another device), GR_E_OOM, GR_E_CUDA, GR_E_TIMEOUT (iteration
 * bound exceeded; the frame's accumulators are then incomplete: reset the
 * frame before rendering into it again). */
gr_status gr_render(gr_scene* const* scenes, int32_t n_scenes, const gr_view_desc* views, int32_t n_views,
                    const gr_render_opts* opts, gr_frame* frame, void* cuda_stream);

/* Device scratch bytes (slot pool, queues, view and order-table descriptors)
 * that gr_render or gr_render_multi of these scenes, views and options would
 * hold in the frame that serves the call; nothing is enqueued.  With
 * opts.pool_size = 0 the default pool depends on the device memory free now
 * (one cudaMemGetInfo).  Errors: as gr_render's argument checks. */
gr_status gr_render_scratch_bytes(gr_scene* const* scenes, int32_t n_scenes, const gr_view_desc* views,
                                  int32_t n_views, const gr_render_opts* opts, size_t* bytes_out);

/* Continuous batching: one render over views whose accumulators live in
 * different frames (e.g. one resident frame per request of a progressive
 * service).  View v adds into view frame_view[v] of frames[v] (shapes must
 * match; no two views may target the same frame view).  The scratch, counters
 * and cached render graph of frames[0] serve the call.  Otherwise as
 * gr_render.  Errors: as gr_render. */
gr_status gr_render_multi(gr_scene* const* scenes, int32_t n_scenes, const gr_view_desc* views, int32_t n_views,
                          const gr_render_opts* opts, gr_frame* const* frames, const int32_t* frame_view,
                          void* cuda_stream);

/* Copy view `view`'s intensity per detector element (Algorithm 1: the sum of
 * the element's sample contributions over their count), float32
 * [height][width][n_bins][n_stokes] (sum / count per bin, 0 where a bin has no
 * samples), to dst (device memory if dst_is_device, else host memory; host
 * copies complete before return).  dst_bytes must be at least the image size.
 * Errors: GR_E_INVALID, GR_E_CUDA. */
gr_status gr_readback(gr_frame* frame, int32_t view, float* dst, size_t dst_bytes, int32_t dst_is_device,
                      void* cuda_stream);

/* Statistics of the last gr_render on this frame (synchronises the stream). */
gr_status gr_frame_stats(gr_frame* frame, void* cuda_stream, gr_stats* out);

/* Inspection of a scene's binary BVH for bit-exact tests (host buffers, may
 * be NULL to query sizes): sorted 64-bit keys (morton << 32 | triangle id) [n],
 * internal nodes (root = 0) as int32 [n-1][2] child references (bit 31 set =
 * leaf slot),
 * and float32 [n-1][12] child boxes (left lo xyz, left hi xyz, right lo, right
 * hi).  Returns the triangle count in *n_out. */
gr_status gr_scene_bvh(gr_scene* scene, int32_t* n_out, uint64_t* keys, int32_t* children, float* boxes);

/* Inspection of the device random stream for bit-exact tests: the raw
 * Philox4x32-10 words of key (seed, view_index) and counters (pixel,
 * sample + i, (segment << 4) | call, 0) for i in [0, n), written to host
 * out_u32 [n][4].  Runs one kernel on the stream and synchronises it. */
gr_status gr_debug_rng(uint32_t seed, uint32_t view_index, uint32_t pixel, uint32_t sample, int32_t segment,
                       int32_t call, int32_t n, uint32_t* out_u32, void* cuda_stream);

/* Inspection of one grating order-table row for precision tests: the weights
 * a_j = J_j(pi h / lambda)^2, j = 0..jmax (Eq. K_grating; h = height_um,
 * lambda = lambda_um), computed and stored exactly as the render stores them
 * in table_dtype (GR_TABLE_F32/F16/BF16: Bessel function in FP64, rounded
 * once to FP32, then to the table type) and decoded back to float, written
 * to host out [jmax + 1].  jmax <= 4096.  Runs one kernel on the stream and
 * synchronises it. */
gr_status gr_debug_order_table(float height_um, double lambda_um, int32_t jmax, int32_t table_dtype, float* out,
                               void* cuda_stream);

/* Inspection of the footprint update for precision tests: for each of the n
 * host quadruples in [n][4] = (beta^2 in um^2, rho, segment length t in m,
 * wavenumber 2 pi / lambda in 1/um) the FP32 update the path applies after a
 * segment (Eq. K_free_space_propagation, zbar = t / |k| with t in um),
 * written to host out [n][2] = (beta^2, rho).  Runs one kernel on the stream
 * and synchronises it. */
gr_status gr_debug_footprint(int32_t n, const float* in, float* out, void* cuda_stream);

/* Footprint-resolved generalized rays through a 1D aperture in a 2D world:
 * the paper's double-slit validation (Sec. 5.1-5.2) with the accurate,
 * footprint-resolved propagation of Sec. 6, at scale.  All lengths in one
 * unit (that of the wavelength); k = 2 pi / lambda.
 *   x0[n_det]        detector element centres on the screen; each element is a
 *                    coherent state of width beta (Eq. wdf_coherent_states)
 *   x_ap, w_ap[n_ap] samples of the aperture plane at distance z from the
 *                    screen: positions and field weights (quadrature weight x
 *                    real field amplitude; the aperture is lit at normal
 *                    incidence), n_ap <= 16384
 *   reach, dtheta    each element's directions theta run from
 *                    atan((x0 - reach)/z) in steps of dtheta up to
 *                    atan((x0 + reach)/z) (exclusive); reach must cover the
 *                    aperture plus the states' width there
 *   rho_cut          truncation radius in units of the propagated width beta'
 *                    (Sec. 6 uses 2.5; a large value disables truncation)
 * Each direction is a generalized ray propagated back over z / cos(theta) in
 * closed form (Eq. K_free_space_propagation from rho = 0: beta'^2 = beta^2 +
 * zbar^2/beta^2, rho' = zbar/beta^2, zbar = z / (k cos(theta))) and overlapped
 * with the aperture field; out[n_det] (host) receives
 * sum_theta |<U_ap, psi_theta>|^2 k cos(theta) dtheta / (2 pi).  Per-direction
 * terms are formed in FP64, the aperture sums in FP32, the per-element sum in
 * FP64 in a fixed order.  *kernel_ms (may be NULL) receives the kernel's device
 * time.  Host buffers; the call synchronises the stream.  GR_E_INVALID for bad
 * sizes or non-positive lengths. */
gr_status gr_aperture_backward_2d(int32_t n_det, const double* x0, int32_t n_ap, const double* x_ap,
                                  const double* w_ap, double beta, double z, double k, double reach, double dtheta,
                                  double rho_cut, double* out, float* kernel_ms, void* cuda_stream);

/* Footprint-resolved generalized rays through a plane aperture in a 3D world:
 * the double-slit validation of Sec. 5.1-5.2 taken to a 2D aperture (any
 * sampled shape, e.g. a rectangle or a disk) and a 2D screen of detector
 * elements, with the accurate propagation and truncation of Sec. 6.  All
 * lengths in one unit (that of the wavelength); k = 2 pi / lambda; the
 * aperture lies in the plane z = 0, lit at normal incidence, the screen in the
 * plane at distance z.
 *   x0[n_det][2]       detector element centres (x, y) on the screen; each is a
 *                      coherent state of width beta (Eq. wdf_coherent_states)
 *   x_ap[n_ap][2], w_ap[n_ap]
 *                      aperture samples: positions and field weights
 *                      (quadrature weight x real field amplitude), n_ap <= 12288
 *   reach, dt          each element's directions t = (s_x, s_y) / s_z form the
 *                      grid (x0 - reach) / z + i dt per axis (i < ceil(2 reach /
 *                      (z dt)) <= 8192), i.e. rays landing on a square grid of
 *                      step z dt over +-reach around the aperture centre; reach
 *                      must cover the aperture plus rho_cut beta'
 *   rho_cut            truncation radius in units of the propagated width beta'
 * Each direction is a generalized ray propagated back over z / s_z in closed
 * form (Eq. K_free_space_propagation from rho = 0), whose footprint is
 * projected obliquely onto the aperture plane (|P d|^2 = |d|^2 - s_z^2 (t.d)^2
 * for an offset d from its landing point), truncated at rho_cut beta' and
 * overlapped with the aperture field; out[n_det] (host) receives
 * sum_t |A|^2 s_z / (pi beta'^2) k^2 s_z^4 dt^2 / (2 pi)^2.  Per-direction terms
 * in FP64, the aperture sums in FP32, the per-element sum in FP64 in a fixed
 * order.  *kernel_ms (may be NULL) receives the kernel's device time.  Host
 * buffers; the call synchronises the stream.  GR_E_INVALID for bad sizes or
 * non-positive lengths. */
gr_status gr_aperture_backward_3d(int32_t n_det, const double* x0, int32_t n_ap, const double* x_ap,
                                  const double* w_ap, double beta, double z, double k, double reach, double dt,
                                  double rho_cut, double* out, float* kernel_ms, void* cuda_stream);

/* ---- Rendering without device allocation (no counterpart in the paper).
 *
 * For callers that must not allocate device memory while rendering: a
 * serving process that sizes all of its GPU memory once at start-up and keeps
 * it under its own allocator, code that runs where an allocation would stall
 * or fail (cudaMalloc and cudaFree synchronise the device; a caching allocator
 * can be empty under memory pressure), or a host framework that forbids
 * libraries from allocating behind its back.  gr_render allocates its
 * wavefront scratch on the stream; gr_render_static runs the same kernels with
 * the scratch in a fixed device array compiled into the library
 * (GR_STATIC_SCRATCH_BYTES; every GPU that loads the library holds it until
 * the process exits) and writes caller-owned accumulators.  It calls no
 * cudaMalloc, cudaFree, event, graph or allocating library routine.
 *
 * scenes/views/opts are as for gr_render (opts.use_graph and opts.profile
 * must be 0).  accum: caller-owned device buffer of 2 * T float32, where T is
 * the sum over views of width * height * n_bins * n_stokes; the first T floats
 * are the per-view sums laid out view after view as [bin][y][x][stokes], the
 * next T their Kahan compensations.  Samples are added (Kahan) into it, so a
 * zeroed buffer gives a fresh image; the mean of a pixel and bin is
 * (sum - compensation) / count, count = number of rendered samples s with
 * s mod n_bins == bin.  The call waits for its work on the stream.
 *
 * Scratch limits: the views' descriptors and grating order tables, plus the
 * slot pool, must fit in GR_STATIC_SCRATCH_BYTES; opts.pool_size (0 = as many
 * slots as fit, about 260k) above that capacity, or descriptors that leave
 * fewer than 256 slots, are rejected with GR_E_INVALID and a message naming
 * the limit.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, which allocates nothing) with the calling thread's
 * device current.  Every call reuses the same array and resets what must
 * start at zero; calls that overlap on the GPU (other streams or threads) race
 * on it and must be serialised by the caller.  Scenes must belong to the
 * current device and accum must be device memory of it (GR_E_INVALID
 * otherwise).  Errors: as gr_render. */
#define GR_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
gr_status gr_render_static(gr_scene* const* scenes, int32_t n_scenes, const gr_view_desc* views, int32_t n_views,
                           const gr_render_opts* opts, float* accum, void* cuda_stream);

/* Thread-local description of the last error (never NULL). */
const char* gr_last_error(void);

/* Library ABI version (this header: 1). */
int32_t gr_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GR_H */
