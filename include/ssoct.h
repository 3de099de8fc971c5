/*
 * ssoct.h - C ABI of libssoct, a single-GPU (sm_103a) implementation of the
 * reconstruction chain of swept-source OCT by off-axis Fresnel-transform digital
 * holography (Charpentier et al., arXiv:2003.08960):
 *
 *   uint16 interferograms I(x, y, t), one per wavelength of a sweep
 *     -> chromatic rescale I'(x, y, t) = I(x lambda_t/lambda_1, y lambda_t/lambda_1, t)   (Eq. 5)
 *     -> discrete Fresnel transform with lambda_1, k_1 for every frame            (Eq. 6)
 *     -> crop to an off-axis window of the hologram plane
 *     -> transform over the sweep (rectangular gate of N_lambda frames)           (Eq. 7)
 *     -> |.|^2 volume and three orthogonal cuts (text after Eq. 7, Fig. 5)
 *
 * Conventions shared by every call
 * - All device pointers are CUDA device memory of the current device, owned by
 *   the caller.  Host pointers are ordinary (pinned or pageable) host memory.
 * - Calls that take a `stream` (a cudaStream_t passed as void*, NULL = legacy
 *   default stream) only enqueue work on it and return; results are ready when
 *   the stream reaches that point.  Statuses are return values; nothing throws.
 * - Layouts are C order.  A frame is uint16 [ny][nx] (x fastest); a stack is
 *   [n][ny][nx].  Volumes are [nlambda][wy][wx] (x fastest) with the depth bin q
 *   unshifted (q = 0 .. nlambda-1).
 * - A plan is not thread-safe; use one plan per host thread or serialise.
 * - lambda_1 is lambda_m[0], the wavelength of the first frame of the sweep
 *   (Eq. 5 and Eq. 6 use it for every frame).
 */
#ifndef SSOCT_H
#define SSOCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SSOCT_API __attribute__((visibility("default")))
#else
#define SSOCT_API
#endif

typedef struct ssoct_plan_s* ssoct_plan;
typedef struct ssoct_batch_s* ssoct_batch;

/* Off-axis window in hologram-plane pixels: columns x0 .. x0+wx-1, rows
 * y0 .. y0+wy-1 of the Nx x Ny hologram computed by Eq. 6.  {0, 0, nx, ny} is
 * the whole plane. */
typedef struct {
  int x0, y0, wx, wy;
} ssoct_window;

typedef enum {
  SSOCT_OK = 0,
  SSOCT_EINVAL = 1,       /* bad argument: size, pointer, alignment, window, index */
  SSOCT_ENOMEM = 2,       /* workspace missing or too small */
  SSOCT_ECUDA = 3,        /* a CUDA runtime call failed (see ssoct_last_error) */
  SSOCT_EAGAIN = 4,       /* reserved */
  SSOCT_ENOTREADY = 5,    /* fewer than nlambda frames pushed since the gate (re)started */
  SSOCT_EDROPPED = 6,     /* a frame sequence number skipped; the gate restarted */
  SSOCT_ETIMEOUT = 7,     /* a kernel gave up waiting on its own work queue */
  SSOCT_EUNSUPPORTED = 8  /* valid request outside the sizes the library is compiled for */
} ssoct_status;

/* Plan flags. */
#define SSOCT_FLAG_MAGNITUDE 0x1u /* volume holds |V| instead of |V|^2 */
/* Eq. 7 on the tensor cores: the sweep-axis DFT as two 16-point stages of
 * tcgen05 MMAs with BF16 hi + lo operands and FP32 accumulation (relative L2
 * error near 1e-5 instead of 1e-7).  nlambda = 256 only (else
 * SSOCT_EUNSUPPORTED at plan creation). */
#define SSOCT_FLAG_TC_AXIAL 0x2u
/* Reserve the workspace of the aberration path (ssoct_set_pupil, ssoct_sharpness):
 * the c P table, one complex frame per wavelength, partial sums.  Any compiled
 * frame size and sweep length (see ssoct_create_plan). */
#define SSOCT_FLAG_PUPIL 0x4u
/* Axial-first order: Eq. 5 and Eq. 7 run first (half spectrum of the real
 * rescaled frames, bins 0..nlambda/2), then Eq. 6 on every depth bin (bins above
 * nlambda/2 from the conjugate planes), whose column pass writes the volume
 * directly.  Eq. 6 is linear and identical for every frame, so V is the same as
 * in the paper's order; HBM traffic drops from 22 to 14 B per voxel.  Frame
 * sizes of the persistent lateral kernel and even nlambda only; no sliding
 * gates, no no-allocation call, not with SSOCT_FLAG_TC_AXIAL (EUNSUPPORTED). */
#define SSOCT_FLAG_AXIAL_FIRST 0x8u

/* Read-only facts about a plan. */
typedef struct {
  int nx, ny, nlambda;
  ssoct_window window;
  double lambda1_m;       /* lambda_1 = lambda_m[0] */
  double dprime_x_m;      /* reconstructed pixel lambda_1 z / (Nx d), Eq. 4 */
  double dprime_y_m;      /* lambda_1 z / (Ny d) */
  double z_b_m;           /* max(Nx, Ny) d^2 / lambda_1: Eq. 6 is meant for z >= z_b (text under Eq. 6) */
  int aliased_chirp;      /* 1 if z < z_b: the input chirp aliases at the frame edge (result still defined) */
  double prefactor_re;    /* K = (i / (lambda_1 z)) exp(-i k_1 z) d^2, the constant of Eq. 6 */
  double prefactor_im;
  size_t workspace_bytes; /* device bytes ssoct_set_workspace needs */
  int ring_slots;         /* frames of lateral scratch kept (L2-resident) */
} ssoct_plan_info_t;

/* Create a plan.  Host only: no CUDA call is made here.
 *   nx, ny     frame size (pixels).  The persistent lateral kernel compiles
 *              nx, ny in {64, 128, 256, 384, 512, 640, 768, 1024} (square),
 *              plus (128, 64) and (64, 128).  Any other pair from that set
 *              (mixed radix 2/3/5) takes a two-pass lateral path
 *              (row pass, column pass through a frame buffer in the
 *              workspace); such plans do not offer ssoct_reconstruct_sliding
 *              or ssoct_reconstruct_frames_noalloc (EUNSUPPORTED there).
 *   nlambda    frames per sweep = depth bins, N_z of Eq. 3 / the gate of Eq. 7.
 *              The library is compiled for {16, 32, 64, 96, 128, 160, 200, 256, 512}.
 *   pitch_m    camera pixel pitch d > 0.
 *   z_m        sensor-to-object distance z != 0 of Eq. 6.
 *   lambda_m   [nlambda] wavelength of each frame of the sweep, > 0; copied.
 *   win        window (NULL = whole plane); must lie inside the frame.
 *   flags      SSOCT_FLAG_*.
 *   out        receives the plan; *out = NULL on error.
 * Builds in float64 and rounds once to float32: per-frame separable linear-
 * interpolation taps (Eq. 5, origin at pixel N/2, taps outside the frame read
 * 0), separable input/output chirps with the centring phase folded in (Eq. 6),
 * FFT twiddles.  EINVAL / EUNSUPPORTED on bad or uncompiled sizes. */
SSOCT_API ssoct_status ssoct_create_plan(int nx, int ny, int nlambda, double pitch_m, double z_m,
                                         const double* lambda_m, const ssoct_window* win,
                                         unsigned flags, ssoct_plan* out);

/* Fill *info.  EINVAL on NULL. */
SSOCT_API ssoct_status ssoct_plan_info(ssoct_plan plan, ssoct_plan_info_t* info);

/* Device workspace size in bytes (tables, frame ring, L2 scratch ring,
 * sweep-axis intermediate, counters). */
SSOCT_API ssoct_status ssoct_workspace_size(ssoct_plan plan, size_t* bytes);
/* The same, under the name of the library's first interface sketch. */
SSOCT_API ssoct_status ssoct_workspace_bytes(ssoct_plan plan, size_t* bytes);

/* Hand the plan caller-owned device memory of at least ssoct_workspace_size
 * bytes, 256-byte aligned.  Uploads the tables (synchronous copy) on the
 * current device, which the plan then uses for every call.  ENOMEM if too
 * small, EINVAL if misaligned or NULL.  The memory must outlive the plan's use. */
SSOCT_API ssoct_status ssoct_set_workspace(ssoct_plan plan, void* dev_ptr, size_t bytes);

/* Append n frames [n][ny][nx] to the plan's ring of nlambda frames (the
 * buffered acquisition of the paper's pipeline).  frames_on_device != 0: the
 * pointer is device memory; otherwise host memory.  Copies are enqueued on
 * `stream` (one cudaMemcpyAsync per contiguous piece).  first_seq >= 0 is the
 * camera sequence number of frames[0]: if it is not the number that follows the
 * previous push, the frames are still stored but the gate restarts with them and
 * EDROPPED is returned, so that no volume mixes frames across a drop (the paper
 * buffers acquisition "to avoid any image drop" for a consistent Eq. 7).
 * first_seq < 0 disables the check.  The frames of a gate must be pushed in
 * sweep order starting at the sweep's first wavelength. */
SSOCT_API ssoct_status ssoct_push_frames(ssoct_plan plan, const uint16_t* frames, int n,
                                         int frames_on_device, int64_t first_seq, void* stream);

/* Reconstruct the volume from the last nlambda pushed frames (ENOTREADY if
 * fewer).  vol_dev: float32 [nlambda][wy][wx] receives |V|^2 (or |V| with
 * SSOCT_FLAG_MAGNITUDE), V being Eq. 7 applied to the windowed Eq. 6 holograms.
 * complex_dev: NULL, or complex64 (interleaved re, im float32) [nlambda][wy][wx]
 * receiving V itself including the prefactor K and the output chirp of Eq. 6.
 * Both 16-byte aligned. */
SSOCT_API ssoct_status ssoct_reconstruct_volume(ssoct_plan plan, float* vol_dev, void* complex_dev,
                                                void* stream);

/* Same, from nlambda frames already in device memory: frames_dev uint16
 * [nlambda][ny][nx], 16-byte aligned, frame t taken at wavelength lambda_m[t].
 * The ring is not touched. */
SSOCT_API ssoct_status ssoct_reconstruct_frames(ssoct_plan plan, const uint16_t* frames_dev,
                                                float* vol_dev, void* complex_dev, void* stream);

/* Same reconstruction as ssoct_reconstruct_frames, for callers that cannot
 * allocate device memory: real-time acquisition code that must not allocate
 * while frames stream in (an allocation can stall the device and drop frames),
 * or plug-ins whose host application owns the device heap.  The paper has no
 * counterpart; it is a deployment variant of the same kernels.
 *   frames_dev, vol_dev, complex_dev: as for ssoct_reconstruct_frames (caller's).
 * The plan needs no workspace.  All other device memory (tables, the lateral
 * kernel's L2 scratch ring and counters, the sweep-axis intermediate) comes from
 * one file-scope device array of 64 MiB that every GPU loading the library keeps
 * until the process exits.  This call allocates nothing (no cudaMalloc, no
 * allocating library routine).  Plans whose workspace would exceed 64 MiB get
 * SSOCT_EUNSUPPORTED with a message saying so (e.g. 256 x 256 x 64 fits,
 * 512 x 512 x 32 does not).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and SM count; make that first call
 * before any stream capture.  Host threads may make their first calls at once
 * (the look-up is done once per device, under a lock).  The address is kept for
 * the life of the process, so after a device reset (cudaDeviceReset) this entry
 * point needs a new process.  Every call shares the array and rewrites the
 * tables and zeroes the counters itself; calls whose work overlaps on the GPU
 * (other streams or host threads) race on it, so serialise them.  A kernel
 * time-out of this call is reported by ssoct_sync on the same plan (SSOCT_ETIMEOUT),
 * provided no other no-allocation call on that device comes in between: the
 * error word lives in the shared array. */
SSOCT_API ssoct_status ssoct_reconstruct_frames_noalloc(ssoct_plan plan, const uint16_t* frames_dev,
                                                        float* vol_dev, void* complex_dev, void* stream);

/* Sliding gates (the paper renders volumes faster than sweeps arrive by
 * sliding the rectangular gate of Eq. 7 along the frame stream).  Requires a
 * periodic sweep: frame i of the stream pushed since the gate (re)started was
 * taken at lambda_m[i mod nlambda], so ring slot r always holds wavelength r.
 * Reconstructs the gate of the last nlambda pushed frames; only frames pushed
 * since the previous sliding call (at most nlambda) go through the lateral
 * stage (Eq. 5 + Eq. 6), their holograms being kept in the sweep-axis
 * intermediate, and the transform over the gate (Eq. 7) runs in slot order.
 * Rotating the gate only multiplies V by exp(2 pi i q s / nlambda), so vol_dev
 * (|V|^2) is that of the gate in time order; complex_dev (NULL or [nlambda][wy]
 * [wx]) receives V in slot order.  Any other reconstruct call on the plan
 * overwrites the intermediate, and the next sliding call redoes all nlambda
 * frames.  ENOTREADY before nlambda frames. */
SSOCT_API ssoct_status ssoct_reconstruct_sliding(ssoct_plan plan, float* vol_dev, void* complex_dev, void* stream);

/* Aberration correction (the paper names it as a use of the phase-resolved
 * volume, introduction; it gives no method).  A phase screen
 * exp(i sum_j c_j Z_j(rho, theta)) multiplies every rescaled frame together with
 * the input chirp of Eq. 6; Z_j are the Noll-ordered Zernike polynomials
 * j = 1..15 (Noll 1976), RMS-normalised on the unit disk, with rho the sensor
 * radius (pixel centre N/2) over min(nx, ny) d / 2, continued outside the disk.
 * Sets the coefficients (radians; coeffs[j - 1] = c_j, ncoeffs 0..15, missing
 * ones 0) and the distance z_m used by ssoct_sharpness (the plan's own z stays
 * in use for the other calls).  Needs SSOCT_FLAG_PUPIL and a workspace.  Host
 * only: the next ssoct_sharpness builds the c P table on the device (FP64
 * phases, one rounding to FP32). */
SSOCT_API ssoct_status ssoct_set_pupil(ssoct_plan plan, const double* coeffs, int ncoeffs, double z_m);

/* Sharpness of the pupil-corrected volume and its gradient, by one forward and
 * one hand-written adjoint pass (all on the device; FP64 sums).  With
 * P_v = |V_v|^2 of Eq. 7 over the window, L = - sum_v P_v^2 / (sum_v P_v)^2.
 * vol_dev [nlambda][wy][wx] (16-byte aligned) receives P.  out_host[17]
 * receives L, dL/dz (per metre, at the z of ssoct_set_pupil) and
 * dL/dc_1 .. dL/dc_15.  Uses the plan's sweep-axis intermediate (like the
 * reconstruct calls, it invalidates the sliding-gate state).  Synchronises
 * `stream`.  ENOTREADY before ssoct_set_pupil. */
SSOCT_API ssoct_status ssoct_sharpness(ssoct_plan plan, const uint16_t* frames_dev, float* vol_dev,
                                       double* out_host, void* stream);

/* Sliding gates for display: the same gate update as ssoct_reconstruct_sliding
 * (new frames through Eq. 5 + Eq. 6 only), then only the three cuts of its
 * |V|^2 instead of the volume: xy[wy][wx] at depth bin z0 as one bin of Eq. 7
 * per pixel, xz[nlambda][wx] at row y0 and yz[nlambda][wy] at column x0 (window
 * coordinates) from Eq. 7 on the tiles that hold them.  Any output may be NULL.
 * While z0 stays the same from call to call, the xy cut is a running sum: the
 * call adds the new frames' holograms and subtracts those they replace (2k
 * slots read per pixel for k new frames instead of nlambda); after nlambda
 * frames swapped in, or when z0, the window contents or the plan's other calls
 * intervene, it is summed over the whole gate again.  The cuts equal
 * ssoct_get_cuts of the sliding volume (xz, yz bit for bit; xy to FP32
 * rounding).  EINVAL if a position lies outside the volume; otherwise as
 * ssoct_reconstruct_sliding. */
SSOCT_API ssoct_status ssoct_sliding_cuts(ssoct_plan plan, int x0, int y0, int z0, float* xy_dev, float* xz_dev,
                                          float* yz_dev, void* stream);

/* The three orthogonal cuts of a volume written by a reconstruct call with this
 * plan (text after Eq. 7; Fig. 5): xy[wy][wx] = P(x, y, z0), xz[nlambda][wx] =
 * P(x, y0, z), yz[nlambda][wy] = P(x0, y, z), coordinates in window pixels and
 * depth bins.  Any output pointer may be NULL to skip that cut.  EINVAL if an
 * index is outside the volume. */
SSOCT_API ssoct_status ssoct_get_cuts(ssoct_plan plan, const float* vol_dev, int x0, int y0, int z0,
                                      float* xy_dev, float* xz_dev, float* yz_dev, void* stream);

/* Wait for `stream` and report what the kernels recorded: ETIMEOUT if a kernel
 * gave up waiting on its work queue (its output is then incomplete), ECUDA on a
 * CUDA error, else OK.  Clears the recorded error.  After a
 * ssoct_reconstruct_frames_noalloc call it reports that call's kernels too. */
SSOCT_API ssoct_status ssoct_sync(ssoct_plan plan, void* stream);

/* Stage timing.  enable != 0: every reconstruct call from now on records CUDA
 * events on its stream around its lateral kernel (Eq. 5 + Eq. 6) and its axial
 * kernel (Eq. 7 + envelope); accumulated times restart at zero.  enable == 0
 * stops recording.  Host only until the next reconstruct call. */
SSOCT_API ssoct_status ssoct_profile(ssoct_plan plan, int enable);

/* Wait for the recorded events and return the summed kernel times (ms) and the
 * number of reconstruct calls recorded since ssoct_profile(plan, 1).  Any output
 * pointer may be NULL. */
SSOCT_API ssoct_status ssoct_profile_read(ssoct_plan plan, double* lateral_ms, double* axial_ms, int* calls);

/* Failure injection for tests of the time-out path.  The next reconstruct calls
 * on this plan start the lateral kernel's work queue `skip` items in, so the
 * items that depend on the skipped ones can never start; every device-side wait
 * gives up after wait_limit_ns (0 = the default of 2 s), the kernels return with
 * their output incomplete, and ssoct_sync reports SSOCT_ETIMEOUT.  Nothing
 * faults or hangs, and the device stays usable.  skip = 0, wait_limit_ns = 0
 * restores normal operation. */
SSOCT_API ssoct_status ssoct_inject_stall(ssoct_plan plan, unsigned skip, unsigned long long wait_limit_ns);

/* Message for the last non-OK status returned on this plan ("" if none). */
SSOCT_API const char* ssoct_last_error(ssoct_plan plan);

/* Name of a status code. */
SSOCT_API const char* ssoct_status_string(ssoct_status s);

/* Release the plan's host memory.  The workspace stays the caller's. */
SSOCT_API void ssoct_destroy_plan(ssoct_plan plan);

/* Autotuner.  Chosen schedule of a plan (see ssoct_autotune). */
typedef struct {
  int lag;         /* steps between a frame's row items and its column items in the lateral kernel's queue */
  int ring_slots;  /* L2 scratch-ring slots in use (<= the workspace's, ring_slots of ssoct_plan_info) */
  int tc_axial;    /* 1: axial pass on the tensor cores (SSOCT_FLAG_TC_AXIAL's form) */
  double ms;       /* measured time of one reconstruction with this choice */
  int from_cache;  /* 1: read from the cache file, nothing timed */
  int candidates;  /* choices timed */
  int axial_first; /* 1: whole-volume reconstructions run the axial-first order (SSOCT_FLAG_AXIAL_FIRST's) */
} ssoct_tune_t;

/* Time the plan's candidate schedules on frames_dev (reconstructing into the
 * scratch volume vol_dev, [nlambda][wy][wx] float) and keep the fastest: the
 * lateral kernel's (lag, ring slots), lag in {1, 2, 3, 4, 6, 8, 12, 16, 24, 32}
 * up to nlambda - 1, each with lag + 2, lag + 4 and all of the workspace's
 * slots (more for smaller frames, whose frames go through the queue faster),
 * times the FP32 and tensor-core axial forms when nlambda is 256, in the paper's order and, where the plan offers it, in the axial-first
 * order (Eq. 5 + Eq. 7 before Eq. 6, the same V; offered when the frame size
 * has the persistent lateral kernel and a width that is a multiple of 64,
 * nlambda is 64, 96, 128, 160, 200 or 256, the plan has no
 * SSOCT_FLAG_PUPIL, and the half-spectrum planes fit in the sweep-axis
 * intermediate, which that order does not use).  A plan made with
 * SSOCT_FLAG_AXIAL_FIRST keeps that order.  An axial-first choice applies to
 * whole-volume reconstructions only: sliding gates and
 * ssoct_reconstruct_frames_noalloc keep the paper's order.  With cache_path (NULL = none), a JSON file holding one entry per line
 * keyed by GPU name, SM count, frame size, sweep length and window is read
 * first (a hit applies the stored choice without timing) and updated after
 * timing.  The choice stays with the plan; results are the same up to the
 * axial form's rounding.  Synchronises `stream`.  EINVAL if the cache cannot be
 * written (the choice is still applied). */
SSOCT_API ssoct_status ssoct_autotune(ssoct_plan plan, const uint16_t* frames_dev, float* vol_dev,
                                      const char* cache_path, void* stream, ssoct_tune_t* result);

/* Batches: several volumes of different sizes (one plan each, e.g. 256^2 x 64
 * up to 1024^2 x 256) reconstructed by one CUDA graph launch.  The paper
 * reconstructs one sweep at a time; batching is this library's.
 * ssoct_batch_create: n distinct plans, each with its workspace set and with
 * profiling and stall injection off (EINVAL otherwise).  lanes = streams the
 * graph spreads the volumes over (volume i on lane i mod lanes; 1 = back to
 * back, 0 = one per volume).  Creates one stream and one event per lane; host
 * memory and CUDA objects are the batch's until ssoct_batch_destroy, the plans
 * stay the caller's and must outlive it. */
SSOCT_API ssoct_status ssoct_batch_create(const ssoct_plan* plans, int n, int lanes, ssoct_batch* out);

/* Reconstruct plan i's sweep frames_dev[i] into vol_dev[i] (as
 * ssoct_reconstruct_frames, no complex output) for all i, ordered after the
 * work already on `stream`; returns without waiting.  The first call on a set
 * of pointers captures all plans' kernels into a graph (on its lanes); later
 * calls on the same pointers relaunch it (one cudaGraphLaunch).  Different
 * pointers recapture. */
SSOCT_API ssoct_status ssoct_batch_run(ssoct_batch b, const uint16_t* const* frames_dev, float* const* vol_dev,
                                       void* stream);

/* Wait for `stream` and report what each plan's kernels recorded (as ssoct_sync). */
SSOCT_API ssoct_status ssoct_batch_sync(ssoct_batch b, void* stream);

/* Number of graph captures so far (-1 for NULL). */
SSOCT_API int ssoct_batch_captures(ssoct_batch b);

/* Description of the last error of a batch call. */
SSOCT_API const char* ssoct_batch_last_error(ssoct_batch b);

/* Release the batch (not its plans). */
SSOCT_API void ssoct_batch_destroy(ssoct_batch b);

#ifdef __cplusplus
}
#endif

#endif /* SSOCT_H */
