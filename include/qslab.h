/*
 * qslab - long-range electrostatics of quasi-2D slabs on one GB300 GPU.
 *
 * C ABI of the SOE-Ewald2D / random-batch SOE-Ewald2D (RBSE2D) long-range
 * path of Gan, Gao, Liang and Xu, "Fast algorithm for quasi-2D Coulomb
 * systems" (arXiv 2403.01521).
 *
 * Problem (Section 2.1, Eqs. 2.1 and 2.8): N point charges q_i at r_i in the
 * slab [0,Lx) x [0,Ly) x [0,Lz], periodic in x and y, free in z, with
 *   U = 1/2 sum_m sum_i sum'_j q_i q_j / |r_i - r_j + (m_x Lx, m_y Ly, 0)|
 * in Gaussian units. Ewald splitting with parameter alpha (Eq. 2.9) gives a
 * short-range part (not computed here) and the long-range part this library
 * computes (Lemma 2.1 minus the self term, Eq. 2.12):
 *   E_long = sum_{k != 0} U^k + U^0 - U_self,
 * with the z-kernels replaced by their sum-of-exponentials (SOE) forms
 * (Eqs. 3.21 and 3.26) and each k handled by sorted forward/backward
 * recursions in z (Eqs. 3.27-3.30, Appendix E). Two ways to sum over k:
 *   - full k-sum over 0 < |k| <= kc (Algorithm 1);
 *   - random batch: P vectors drawn i.i.d. from h(k) ~ e^{-k^2/(4 alpha^2)}
 *     on the whole lattice, weighted by H/P (Eqs. 4.5-4.9, Algorithm 2).
 * The k = 0 term is always computed exactly (in its SOE form).
 *
 * Outputs, for every particle: the long-range potential phi_i (including the
 * j = i constants, so that E_long = 1/2 sum_i q_i phi_i and dE/dq_i = phi_i)
 * and the long-range force F_i = -dE_long/dr_i.
 *
 * Conventions shared by all calls:
 *   - Return value 0 on success, a negative QSLAB_ERR_* code otherwise.
 *     qslab_strerror() gives a message. A failed call changes no
 *     configuration, no random-batch counter and no output; a failed device
 *     allocation may leave the context without its workspace (allocated
 *     again by the next call), which ends the state an energy-only call left
 *     for qslab_compute_adjoint().
 *   - A context belongs to one host thread at a time and to one CUDA device
 *     (chosen at creation; every call makes it current).
 *   - Device pointers are plain CUDA device addresses (for example from
 *     torch.Tensor.data_ptr()); the caller owns them. The library owns its
 *     workspace, allocated on first use and grown as needed, and frees it in
 *     qslab_destroy().
 *   - Work is ordered on the caller's stream (cudaStream_t passed as void*;
 *     NULL = legacy default stream). qslab_compute() does not synchronise.
 *     Parts of a call that do not depend on each other (the k = 0 term, the
 *     mode table, the real-space part of an MD force pass) run on internal
 *     streams of the context, forked from the caller's stream and joined
 *     back to it with events before the call's last kernel, so the call as a
 *     whole stays ordered on that stream and can be captured in a CUDA graph.
 */
#ifndef QSLAB_H
#define QSLAB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qslab_ctx qslab_ctx;

/* Precision of positions, charges, potentials and forces, and of the
 * arithmetic. QSLAB_FP64: everything in FP64. QSLAB_FP32C (compensated
 * FP32): FP32 inputs and outputs; FP32 phases and FP32 recurrences within
 * each chunk of sorted particles (the k != 0 scans and the k = 0 scans of
 * the exponential sums); the k != 0 chunk aggregates (up to 12 SOE pair
 * representatives) as tensor-core TF32 products of split operands
 * (x = x_hi + x_lo) with FP32 accumulation, at FP32-level accuracy;
 * double-float (two FP32 numbers, about 48 bits) chunk-to-chunk carries,
 * and double-float prefix sums of q and q z for the |z| part of the k = 0
 * term; the per-particle sums over mode ranges, the j = i constants and the
 * energy reduction in double-float (in FP64 when charged walls are set). */
#define QSLAB_FP64 0
#define QSLAB_FP32C 1

#define QSLAB_OK 0
#define QSLAB_ERR_INVALID_ARG (-1)    /* bad argument or unsupported size    */
#define QSLAB_ERR_NOT_CONFIGURED (-2) /* box, alpha, SOE or k-set missing    */
#define QSLAB_ERR_NONFINITE (-3)      /* NaN or Inf in positions or charges  */
#define QSLAB_ERR_Z_OUT_OF_RANGE (-4) /* some z outside [0, Lz]              */
#define QSLAB_ERR_NONNEUTRAL (-5)     /* |sum q| above tolerance (Thm 2.1)   */
#define QSLAB_ERR_ALLOC (-6)          /* device or host allocation failed    */
#define QSLAB_ERR_CUDA (-7)           /* a CUDA runtime call failed          */
#define QSLAB_ERR_TIMEOUT (-8)        /* a bounded device wait gave up (the
                                         z-sort's look-back between CTAs);
                                         the call's outputs are unspecified */
#define QSLAB_ERR_TOO_LARGE (-9)      /* exceeds qslab_compute_static's scratch */
#define QSLAB_ERR_INTERNAL (-10)      /* debug build: an internal index check
                                         failed (a library bug, not an input
                                         error); the release build never
                                         returns it */

/* Create a context on CUDA device `cuda_device` with precision `prec`
 * (QSLAB_FP64 or QSLAB_FP32C). *out receives the handle. */
int qslab_create(qslab_ctx** out, int cuda_device, int prec);

/* Release the context and all its device memory. NULL is ignored. */
void qslab_destroy(qslab_ctx* ctx);

/* Box lengths (Section 2.1): x in [0,Lx), y in [0,Ly) (taken modulo the
 * box), z in [0, Lz]. All must be finite and > 0. */
int qslab_set_box(qslab_ctx* ctx, double Lx, double Ly, double Lz);

/* Ewald splitting parameter alpha > 0 (Eq. 2.9). */
int qslab_set_alpha(qslab_ctx* ctx, double alpha);

/* Full k-sum (Algorithm 1): every k = 2 pi (m_x/Lx, m_y/Ly) != 0 with
 * (2 pi m_x/Lx)^2 + (2 pi m_y/Ly)^2 <= kc^2. Selects the full-k mode. */
int qslab_set_kcut(qslab_ctx* ctx, double kc);

/* Random batch (Section 4.1, Algorithm 2): each qslab_compute() draws P
 * lattice vectors i.i.d. from h(k) (origin excluded) with a counter-based
 * generator keyed by `seed`; the counter starts at 0 and advances by one per
 * call. Selects the random-batch mode. 1 <= P <= 65536. */
int qslab_set_rbe(qslab_ctx* ctx, int P, uint64_t seed);

/* SOE of the Gaussian, e^{-x^2} ~ sum_l w_l e^{-s_l |x|} (Eqs. 3.1, 3.6):
 * M complex nodes s and weights w given as real/imaginary host arrays of
 * length M (copied). Requirements: 1 <= M <= 32, Re s_l > 0, and the set is
 * closed under complex conjugation (a real node is its own conjugate). */
int qslab_set_soe(qslab_ctx* ctx, int M, const double* s_re, const double* s_im,
                  const double* w_re, const double* w_im);

/* Neutrality tolerance: compute() flags QSLAB_ERR_NONNEUTRAL when
 * |sum q| > tol * sum |q|. Default 64 x the unit roundoff of the precision.
 * A negative tol disables the check. With charged walls
 * (qslab_set_walls) the check covers particles and walls together:
 * |sum q + A (sigma_bot + sigma_top)| > tol (sum |q| + A (|sigma_bot| + |sigma_top|)),
 * A = Lx Ly of the slab. */
int qslab_set_neutrality_tol(qslab_ctx* ctx, double tol);

/* Launch shape: particles per chunk (0 = automatic; at most 512 for FP32C,
 * 256 for FP64) and modes per CTA (0 = automatic; a multiple of 32, at most
 * 256). Results do not depend on it beyond rounding. */
int qslab_set_tuning(qslab_ctx* ctx, int chunk, int modes_per_cta);

/* Arithmetic throughput of the device (the paper has no counterpart; it
 * gives the measured ceilings against which the k-space kernels' FP32
 * arithmetic is judged). Runs four microbenchmark kernels on `stream` over
 * 8 blocks per SM, each thread 16 independent dependency chains, timed with
 * CUDA events (best of 3 after one warm-up), and writes lane operations per
 * second to out4 (host, 4 doubles): [0] scalar FP32 FMA, [1] packed two-wide
 * FP32 FMA (__ffma2_rn, counted as two), [2] FP64 FMA, [3] ex2.approx.f32.
 * Allocates and frees a few KB of device memory; synchronises the stream. */
int qslab_measure_peaks(int cuda_device, double* out4, void* stream);

/* Launch-shape autotuner (the paper has no counterpart; the launch shape
 * changes no result beyond rounding). Times qslab_compute_batched() on the
 * given replicas (R = 1, offsets {0, N} and boxes = the context's box for a
 * single slab) for every candidate pair (chunk length 64..512, modes per CTA
 * 64..256 or automatic), reps timed calls each after one warm-up call, with
 * CUDA events on `stream`, and keeps the fastest with qslab_set_tuning().
 *   pos, q     device inputs as for qslab_compute_batched(); read only
 *   reps       timed calls per candidate, 1..100
 *   chunk, modes_per_cta   receive the chosen tuning (either may be NULL)
 * The random-batch counter is restored afterwards: tuning draws no samples
 * from the user's sequence. Synchronises the stream; allocates the largest
 * workspace among the candidates (candidates that do not fit are skipped).
 * Returns the status of the tuning calls (a device-side input error aborts
 * the tuning and leaves the previous tuning in place). */
int qslab_autotune(qslab_ctx* ctx, int R, const int64_t* offsets,
                   const double* boxes, const void* pos, const void* q,
                   void* stream, int reps, int* chunk, int* modes_per_cta);

/* Long-range energy, potentials and forces (Algorithm 1 steps 4-5, 7-9, or
 * Algorithm 2 steps 4-7, 9; the real-space part is not included).
 *   N       number of particles, 1 <= N <= 2^31 - 1
 *   pos     device, N x 3 row-major (x, y, z), double (FP64) or float (FP32C)
 *   q       device, N charges, same type
 *   energy  device, one double (always FP64), or NULL
 *   phi     device, N potentials (same type as pos), or NULL
 *   force   device, N x 3 forces (same type as pos), or NULL
 *   stream  cudaStream_t or NULL
 * Host-side argument errors are returned at once. Input errors found on the
 * device (NONFINITE, Z_OUT_OF_RANGE, NONNEUTRAL) are recorded in the
 * context's status word and returned by qslab_last_status(); the outputs of
 * such a call are unspecified. */
int qslab_compute(qslab_ctx* ctx, int64_t N, const void* pos, const void* q,
                  double* energy, void* phi, void* force, void* stream);

/* Many independent slabs ("replicas") in one call: the same computation as
 * qslab_compute() for each replica, batched into one launch sequence (every
 * kernel covers all replicas; no launch per replica). The paper treats one
 * slab at a time; this is the same method applied to R of them at once.
 *   R        number of replicas, 1 <= R <= 2^20
 *   offsets  host, R + 1 int64: replica r owns particles
 *            [offsets[r], offsets[r+1]) of pos, q, phi and force;
 *            offsets[0] = 0, non-decreasing (empty replicas allowed),
 *            1 <= offsets[R] <= 2^31 - 1
 *   boxes    host, R x 3 doubles (Lx, Ly, Lz) per replica; the box set by
 *            qslab_set_box() is not used
 *   energies device, R doubles (FP64), or NULL: the energy of each replica
 *   pos, q, phi, force, stream: as for qslab_compute(), over all particles
 * alpha, the SOE and the k-set (k cutoff, or P and seed) are the context's
 * and are shared by all replicas; the full k-sum uses each replica's own
 * half-plane lattice, the random batch draws P vectors per replica from the
 * replica's own h(k), with the stream index r in the generator's counter.
 * Every replica must be charge neutral on its own (with the walls, if set).
 * Tables derived from offsets and boxes are cached in the context: calls
 * that repeat them do no host-side set-up and no synchronous transfer. Such a
 * repeat call (after one ordinary call with the same arguments and buffers
 * has sized the context) issues only stream-ordered work and may be captured
 * in a CUDA graph; a graph replay recomputes everything, including a fresh
 * random-batch sample. Device-side input errors go to the status word as for
 * qslab_compute(). */
int qslab_compute_batched(qslab_ctx* ctx, int R, const int64_t* offsets,
                          const double* boxes, const void* pos, const void* q,
                          double* energies, void* phi, void* force,
                          void* stream);

/* Energy only, and its adjoint (Section 3.2's recursion run forward for
 * the energy; the gradient by the bidirectional scans of Appendix E run
 * afterwards, on demand).
 * qslab_compute_energy(): the long-range energy of qslab_compute() (same
 * sort, k-set, sample and k = 0 term) from forward sums only: per mode the
 * pair energy gam Re sum_beta c_beta sum_i conj(u_i) sum_{j<i} u_j
 * e^{-beta (z_i - z_j)} (each pair once), without the per-particle gather;
 * about half the work of the full call.
 *   energy   device, one double (required)
 *   N, pos, q, stream: as for qslab_compute()
 * The call leaves the sorted order, the chunk carries of both directions,
 * the mode tables (including the random-batch sample) and the k = 0 term in
 * the context's workspace.
 * qslab_compute_batched_energy(): the same for R replicas (arguments as
 * for qslab_compute_batched(); energies required).
 * qslab_compute_adjoint(): the gradient of that energy, from what the last
 * energy-only call left: phi_i = dE/dq_i and F_i = -dE/dr_i (device, the
 * precision's type, N and N x 3 in the caller's order of that call; either
 * may be NULL, not both), by the bidirectional recurrences over the stored
 * sorted order with the phases recomputed. Equal to the phi and force of
 * qslab_compute() on the same inputs and sample. It must follow the
 * energy-only call on the same stream (or after it completed), with no other
 * long-range call, MD step or configuration change on the context in
 * between; otherwise it returns QSLAB_ERR_NOT_CONFIGURED. It may be called
 * more than once. */
int qslab_compute_energy(qslab_ctx* ctx, int64_t N, const void* pos, const void* q,
                         double* energy, void* stream);
int qslab_compute_batched_energy(qslab_ctx* ctx, int R, const int64_t* offsets,
                                 const double* boxes, const void* pos, const void* q,
                                 double* energies, void* stream);
int qslab_compute_adjoint(qslab_ctx* ctx, void* phi, void* force, void* stream);

/* Virial tensor of the long-range energy, for pressures in the NPT ensemble
 * (Section 4.3: the random-batch dynamics extends to NPT through the virial;
 * Section 2.4: the L_z-dependent constant of the particle-slab potential of
 * Thm 2.4 is what the walls' part needs). The same call as qslab_compute()
 * (energy, phi, force as there) that also returns
 *   W_ab = -dE_long/d eps_ab,   virial = (W_xx, W_yy, W_zz, W_xy, W_xz, W_yz),
 * for the strain r -> (I + eps) r applied to the particles, to the lateral
 * lattice vectors and to the charged walls (which keep their charge per cell,
 * so sigma scales as 1/A; the top wall at z = L_z moves with the box).
 * eps_zx = eps_zy = 0 keeps the lattice in the plane z = 0, and W_yx = W_xy
 * (rotation invariance in the plane). In detail:
 *   lateral: W_ab = delta_ab (E + U_self) + sum_k (k_a k_b/|k|) dU^k/d|k|,
 *            U^k of the SOE kernel (Eq. 3.21) over the k-set of the call
 *            (random batch: each sample weighted as in Eq. 4.7, an unbiased
 *            estimate of the full sum), plus the walls' modes;
 *   zz, xz, yz: sum_i F_i,a z_i plus the top wall's explicit terms.
 * The pressure tensor is P_ab = (sum_i m v_a v_b + W_ab)/(Lx Ly Lz) once
 * the real-space virial (qslab_compute_realspace_virial) is added.
 *   energy, force  required (device; the z-components are formed from force)
 *   phi            device or NULL
 *   virial         device, 6 doubles (FP64)
 * Needs more workspace than qslab_compute() (about 40 bytes per chunk and
 * mode); errors as for qslab_compute(). */
int qslab_compute_virial(qslab_ctx* ctx, int64_t N, const void* pos, const void* q,
                         double* energy, void* phi, void* force, double* virial,
                         void* stream);

/* qslab_compute_batched() with the virial of every replica:
 *   energies, force  required (device)
 *   virial           device, R x 6 doubles, the order of qslab_compute_virial() */
int qslab_compute_batched_virial(qslab_ctx* ctx, int R, const int64_t* offsets,
                                 const double* boxes, const void* pos, const void* q,
                                 double* energies, void* phi, void* force,
                                 double* virial, void* stream);

/* The same computation from host buffers: copies pos and q (host, layout as
 * above; pinned memory makes the copies asynchronous) to the device, runs,
 * copies energy/phi/force back to host buffers (any may be NULL) and waits
 * for the stream. Returns the call's full status, including device-side
 * input errors. */
int qslab_compute_host(qslab_ctx* ctx, int64_t N, const void* pos_host,
                       const void* q_host, double* energy_host,
                       void* phi_host, void* force_host, void* stream);

/* The same computation as qslab_compute(), for callers that cannot allocate
 * device memory when they need the result (inside another framework's memory
 * pool, under a fixed device-memory budget, or in a time step where an
 * allocation and the synchronisation it may bring are not allowed). It calls
 * no cudaMalloc, cudaFree or other allocating routine: all scratch comes from
 * one 64 MiB array in device memory that the library defines at file scope
 * and that every GPU loading the library holds until the process exits.
 * The paper has no counterpart; this is an interface variant only.
 *   - Arguments, layouts and results as for qslab_compute(); the context must
 *     be configured. Its own device buffers are not used; the mode and
 *     sampler tables are copied into the array on every call, in the call's
 *     stream order (the mode list, the sampling distribution and the per-box
 *     constants are reused on the host while the configuration and the box
 *     stay the same; no device allocation).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress), once per device.
 *   - Limits: the tables must fit 8 MiB and the workspace the remaining
 *     56 MiB (at P = 200 random-batch modes about 1.7e5 particles in FP32C);
 *     larger problems return QSLAB_ERR_TOO_LARGE before any device work.
 *   - Every call uses the same array and it keeps the previous call's
 *     contents (what must start at zero is cleared by the call). Calls that
 *     overlap on the GPU (two streams, or two contexts on one device) race on
 *     it: serialise them.
 *   - The call waits for its stream and returns the full status, including
 *     device-side input errors; the random-batch counter advances as for
 *     qslab_compute() (qslab_get_sampled_modes() does not see these samples). */
int qslab_compute_static(qslab_ctx* ctx, int64_t N, const void* pos, const void* q,
                         double* energy, void* phi, void* force, void* stream);

/* Random-batch k-sampler (Section 4, App. G). QSLAB_SAMPLER_IID (default):
 * P independent draws from h(k) by inversion of its two one-dimensional
 * factors. QSLAB_SAMPLER_METROPOLIS: the independence Metropolis chain of
 * App. G: proposals are rounded normals of variance (alpha L)^2/(2 pi^2)
 * per axis (Box-Muller from Philox4x64-10 words), the origin is rejected,
 * other proposals are accepted with probability
 * min{1, H(new) q(old)/(H(old) q(new))}; each call runs a fresh chain of
 * P * thin steps per slab (started at the first proposal that is not the
 * origin) and keeps every thin-th state (the downsampling rate, 1..4096).
 * Both samplers weight every sample by H/P (Eq. 4.7) and draw from the
 * counter of the call, so CUDA-graph replays draw fresh samples. Takes
 * effect at the next random-batch call; QSLAB_ERR_INVALID_ARG for another
 * kind or thin. */
#define QSLAB_SAMPLER_IID 0
#define QSLAB_SAMPLER_METROPOLIS 1
int qslab_set_rbe_sampler(qslab_ctx* ctx, int kind, int thin);

/* Charged walls at z = 0 (bottom) and z = Lz (top), Section 2.4. The walls
 * carry doubly periodic surface charge densities (charge per unit area)
 *   sigma_bot(rho) = sigma_bot + sum_w 2 Re[(bot[2w] + i bot[2w+1]) e^{i k_w.rho}]
 *   sigma_top(rho) = sigma_top + sum_w 2 Re[(top[2w] + i top[2w+1]) e^{i k_w.rho}]
 * with k_w = (2 pi mxy[2w]/Lx, 2 pi mxy[2w+1]/Ly), w < nw. After this call
 * qslab_compute() and qslab_compute_batched() (every replica, each with its
 * own box) add the particle-slab potential of Thm 2.4,
 *   phi_p-s(r) = -2 pi [sigma_bot z + sigma_top (Lz - z)]
 *                + sum_w Re[e^{i k_w.rho} (4 pi / |k_w|)
 *                       ((bot_w) e^{-|k_w| z} + (top_w) e^{-|k_w| (Lz - z)})],
 * to phi, its force -q grad phi_p-s to force, and sum_i q_i phi_p-s(r_i) to
 * the energy (each particle-wall pair counted once, so that F = -grad E and
 * phi = dE/dq still hold). The particles then need not be neutral; the
 * neutrality check covers particles and walls together.
 *   sigma_bot, sigma_top: uniform parts (finite).
 *   nw: 0 (uniform walls, the special case after Thm 2.4) to 64 Fourier modes.
 *   mxy: host int32 [nw][2], (mx, my) != (0, 0), |mx|, |my| <= 2^20, each
 *        pair (m, -m) listed at most once; bot, top: host double [nw][2]
 *        (real, imaginary part). Copied; may be NULL when nw = 0.
 * QSLAB_ERR_INVALID_ARG on any violation (the walls are then unchanged).
 * qslab_clear_walls() removes them. The real-space part does not involve
 * the walls. */
int qslab_set_walls(qslab_ctx* ctx, double sigma_bot, double sigma_top, int nw,
                    const int32_t* mxy, const double* bot, const double* top);
int qslab_clear_walls(qslab_ctx* ctx);

/* Real-space cut-off rc for qslab_compute_realspace() (Section 2.3:
 * pairs with |r_ij + M| > rc are dropped; the truncation error is of order
 * erfc(alpha rc)). */
int qslab_set_rcut(qslab_ctx* ctx, double rc);

/* The real-space part of the Ewald2D splitting (Eq. 2.10): per particle
 *   phi_s,i = sum_{j, M} q_j erfc(alpha |r_ij + M|)/|r_ij + M|   (j != i when M = 0)
 * over the images M = (mx Lx, my Ly, 0) with |r_ij + M| <= rc, its forces
 * F_i = -dE_s/dr_i and E_s = 1/2 sum_i q_i phi_s,i. Adding it to
 * qslab_compute()'s long-range part gives the total Coulomb energy, potential
 * and forces of the slab (Eq. 2.9). Uses the context's box, alpha, rc and
 * precision (not the k-set).
 *   N, pos, q, energy, phi, force, stream: as for qslab_compute(); the outputs
 *   are written, not added to. energy (device double), phi and force may be
 *   NULL.
 * Needs rc <= min(Lx, Ly)/3 (QSLAB_ERR_INVALID_ARG otherwise) and rc set
 * (QSLAB_ERR_NOT_CONFIGURED). Device-side input errors (non-finite values,
 * z outside [0, Lz]) go to the status word as for qslab_compute(). Cell list
 * with cells of edge >= rc/2; every pair is evaluated from both ends, in a
 * fixed order (bitwise reproducible). Own workspace: it may run on another
 * stream than the long-range call of the same context. The paper evaluates
 * this part with a cell or Verlet list (Section 2.3); not part of Algorithms
 * 1 and 2's long-range path. */
int qslab_compute_realspace(qslab_ctx* ctx, int64_t N, const void* pos, const void* q,
                            double* energy, void* phi, void* force, void* stream);

/* qslab_compute_realspace() that also returns the pair virial of the
 * real-space sum (Eq. 2.10 within rc), for pressures (Section 4.3):
 *   W_ab = 1/2 sum_{i, j, M} (F_ij)_a (r_ij + M)_b,
 * F_ij the force on i from the pair term of j, as
 * virial = (W_xx, W_yy, W_zz, W_xy, W_xz, W_yz) (device, 6 doubles, FP64
 * sums). With qslab_compute_virial() it gives the virial of the whole
 * Ewald2D energy, whose trace equals that energy (the Coulomb energy is
 * homogeneous of degree -1 in all lengths). Other arguments and errors as for
 * qslab_compute_realspace(); virial must not be NULL. */
int qslab_compute_realspace_virial(qslab_ctx* ctx, int64_t N, const void* pos, const void* q,
                                   double* energy, void* phi, void* force, double* virial,
                                   void* stream);

/* Langevin dynamics of one slab (Section 4.3) with the forces of this
 * library: the long-range part as configured (full k-sum or random batch,
 * either sampler, charged walls if set), the real-space part within rc, and
 * the short-range model of Section 5.2: a shifted-truncated Lennard-Jones
 * repulsion 4 eps [(s/r)^12 - (s/r)^6 + 1/4] for r < 2^(1/6) s between
 * particles (lj_eps, lj_sigma; 2^(1/6) lj_sigma <= rc) and in the distance
 * to each wall (wall_eps, wall_sigma). lj_eps = 0 or wall_eps = 0 turns a
 * term off. Time stepping is BAOAB (Leimkuhler and Matthews 2013) in
 * velocities: v += dt/2 F/m; x += dt/2 v; v <- c1 v + c2 xi with
 * c1 = e^{-gamma dt/m}, c2 = sqrt((1 - c1^2) kT/m); x += dt/2 v; new F;
 * v += dt/2 F/m. x and y are wrapped into [0, L). The noise xi of particle
 * i at step n comes from Philox4x64-10 with counter (i, n, 0, 0x4D445331)
 * and key (seed, 0) through the Box-Muller transform; n is a device counter
 * advanced by every step (so CUDA-graph replays continue the noise), read
 * and set with qslab_md_get_step / qslab_md_set_step. */
int qslab_md_configure(qslab_ctx* ctx, double dt, double mass, double gamma, double kT,
                       double lj_eps, double lj_sigma, double wall_eps, double wall_sigma,
                       uint64_t seed);
/* The total force at pos into force (device, 3N of the context's
 * precision), and if energies (device double[4]) is not NULL: the
 * long-range energy (walls included), the real-space energy with the LJ
 * pairs, the LJ wall energy and the kinetic energy of vel (vel may be
 * NULL: 0). Needs qslab_md_configure, the box and rc
 * (QSLAB_ERR_NOT_CONFIGURED). Stream-ordered: the real-space part runs on
 * an internal stream of the context, forked from `stream` and joined back
 * to it with events (so it overlaps the long-range call and can be captured
 * in a CUDA graph together with it). */
int qslab_md_forces(qslab_ctx* ctx, int64_t N, const void* pos, const void* q, void* vel,
                    void* force, double* energies, void* stream);
/* nsteps >= 1 BAOAB steps in place: pos, vel (device, 3N) and force (the
 * total force at pos on entry, as left by qslab_md_forces or the previous
 * step; updated). energies as for qslab_md_forces, after the last step.
 * No allocation once the buffers for N exist (first call), so a call can be
 * captured in a CUDA graph. Device-side input errors go to the status word;
 * a particle leaving [0, Lz] sets QSLAB_ERR_Z_OUT_OF_RANGE. */
int qslab_md_step(qslab_ctx* ctx, int64_t N, void* pos, void* vel, const void* q, void* force,
                  int nsteps, double* energies, void* stream);
int qslab_md_set_step(qslab_ctx* ctx, uint64_t step);
int qslab_md_get_step(qslab_ctx* ctx, uint64_t* step);

/* Random-batch mode: copy the lattice vectors used by the latest
 * qslab_compute() or qslab_compute_batched() into mxy (host, 2*P*R int32:
 * (m_x, m_y) pairs, replica by replica; R = 1 after qslab_compute()) and, if
 * weight is not NULL, the sample weights H_r/P (R doubles). Synchronises
 * the context's stream. */
int qslab_get_sampled_modes(qslab_ctx* ctx, int32_t* mxy, double* weight);

/* Generator state (seed, number of random-batch compute calls made), for
 * bit-exact resumption of a random-batch sequence. The counter lives in
 * device memory and is advanced on the stream by every call (so that a call
 * replayed from a CUDA graph draws a fresh sample); both functions
 * synchronise the stream of the latest call. */
int qslab_get_rng_state(qslab_ctx* ctx, uint64_t* seed, uint64_t* counter);
int qslab_set_rng_state(qslab_ctx* ctx, uint64_t seed, uint64_t counter);

/* Number of k vectors summed per call: half-plane count for the full k-sum
 * (each stands for k and -k), P for the random batch. */
int qslab_num_modes(qslab_ctx* ctx);

/* Wait for the stream of the latest compute() and return its device-side
 * status (QSLAB_OK or the first input error), then clear it. */
int qslab_last_status(qslab_ctx* ctx);

/* Per-phase timings of the latest compute(), measured with CUDA events on its
 * stream while timing is enabled (qslab_set_timing(ctx, 1)). ms8 receives, in
 * milliseconds: [0] checks + z-sort + gather, [1] the wait for the mode
 * table (sampler and coefficients; built on an internal stream concurrently
 * with [0], so this is the part that [0] does not cover), [2] k-space chunk aggregates, [3] carries, [4] k-space recurrences with the
 * gather, [5] k = 0 term (it runs on an internal stream concurrently with
 * [1]-[4]), [6] combine + energy, [7] total. *launches (may be NULL)
 * receives the number of kernels the call launched. Synchronises. */
int qslab_set_timing(qslab_ctx* ctx, int enable);
int qslab_get_timings(qslab_ctx* ctx, double* ms8, int* launches);

/* Message for a return code. */
const char* qslab_strerror(int code);

/* Diagnostics (the paper has no counterpart; for tests of the library's
 * own error handling).
 * qslab_debug_alloc_count(): the number of device allocations (cudaMalloc)
 * the library has made in this process, over all contexts.
 * qslab_debug_fail_alloc(n): the next n device allocations of the library
 * fail as an out-of-memory cudaMalloc would, decided on the host without
 * calling the CUDA runtime (no GPU fault); n = 0 turns this off. A call
 * whose allocation fails returns QSLAB_ERR_ALLOC. When growing a buffer the
 * library allocates the new one before releasing the old one; if that
 * fails it releases the old buffer and tries once more (so one injected
 * failure is absorbed, two fail the call). */
long long qslab_debug_alloc_count(void);
int qslab_debug_fail_alloc(int n);
/* qslab_debug_stall_sort(tile): in the next long-range call (of any
 * context in this process) the z-sort's first digit pass leaves tile
 * `tile` (4096 keys each, in order) without its published counts, so that
 * the next tile's bounded wait runs out (about 0.1 to 1 s): the call then
 * completes with QSLAB_ERR_TIMEOUT in the status word and unspecified
 * outputs, and the context stays usable. Applies only to calls with more
 * than 2048 particles (smaller sorts run in one CTA and do not wait). */
int qslab_debug_stall_sort(int tile);

#ifdef __cplusplus
}
#endif
#endif /* QSLAB_H */
