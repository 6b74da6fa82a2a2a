/*
 * bude.h -- C ABI of the GB300 (sm_103a) pose-energy library libbude.so.
 *
 * The library evaluates the per-pose protein-ligand docking energy that the
 * miniBUDE "fasten" kernel computes (arxiv 2509.21039, Sec. 2.2, Listing 4; FLOP
 * count Eq. 3): every pose moves the ligand rigidly (three angles, three
 * translations), every ligand x protein atom pair is scored by steric,
 * electrostatic and desolvation terms looked up by atom-type pair, and half
 * the sum is the pose energy.  The paper does not write the forcefield down;
 * the pair energy used here is, with R = r_a + r_b, H = (h_a + h_b)/2,
 * Q = q_a q_b, s = d - R and phi(u) = clamp-to-[0,1] cubic (1-u)^2 (1+2u):
 *
 *   e = H (s/R)^2 [s<0] + 4 Q w phi(s/4) + S phi(s/2)
 *
 * where w = 2 for a donor-acceptor pair (else 1) and S = 1/2 when exactly one
 * atom of the pair is polar (hbtype != 0), else 0.  All terms vanish for
 * d >= R + 4 Angstrom.
 *
 * Conventions shared by every call
 *  - Pointers named "device" must be CUDA device (or managed) memory of the
 *    current device; the library never dereferences them on the host.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Compute calls are asynchronous on it and never synchronise,
 *    except where a call says otherwise.
 *  - Every call returns BUDE_OK (0) or a negative BUDE_ERR_* code and never
 *    aborts, asserts or traps.  bude_status_string() names a code;
 *    bude_last_error() gives a one-line message for the last failure on the
 *    calling thread.
 *  - Calls that use the same deck (or the same batch plan) must not overlap
 *    on the GPU: they share the deck's scratch workspace.
 */
#ifndef BUDE_H
#define BUDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define BUDE_API __attribute__((visibility("default")))
#else
#define BUDE_API
#endif

#define BUDE_OK 0
#define BUDE_ERR_INVALID_ARG (-1) /* null pointer, bad size, type or option */
#define BUDE_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define BUDE_ERR_OOM (-3)         /* device allocation failed */
#define BUDE_ERR_UNSUPPORTED (-4) /* shape or option outside what is built */
#define BUDE_ERR_DEVICE_FLAG (-5) /* a device-side check raised its error word */

/* Arithmetic variants of the energy kernels. */
#define BUDE_FP32_IEEE 0 /* FP32, correctly rounded sqrt/div, no flush-to-zero */
#define BUDE_FP32_FAST 1 /* FP32, approximate sqrt and sin/cos, flush-to-zero */
#define BUDE_FP32_COMP 2 /* as IEEE, each ligand atom's FP32 sum folded in FP64 */
#define BUDE_FP64 3      /* every operation in FP64 */

/* Limits of the library. */
#define BUDE_MAX_TYPES 1024

/*
 * Deck description: the three inputs of Listing 4 besides the poses.
 * Atom records are 16 bytes, {x, y, z, type}, the type being an int32 stored
 * in the fourth 4-byte word (Sec. 2.2 describes the same flattening of the
 * Atom struct to four 4-byte fields).  Forcefield rows are
 * {radius, hardness, elsc, hbtype} with hbtype an int32 in the fourth word
 * (0 none, 1 donor, 2 acceptor).
 */
typedef struct {
    int32_t n_lig;          /* ligand atoms, >= 0 */
    int32_t n_pro;          /* protein atoms, >= 0 */
    int32_t n_types;        /* forcefield rows, 1..BUDE_MAX_TYPES */
    const float* lig_xyzt;  /* device, [n_lig][4] */
    const float* pro_xyzt;  /* device, [n_pro][4] */
    const float* ff;        /* device, [n_types][4] */
} bude_deck_desc;

/*
 * Launch options.  Zero in any field selects the library default for the
 * variant (the defaults come from the autotuner's tables compiled in or set
 * with bude_set_default_options).  The defaults are one shape per variant,
 * shared by all calls: a gradient call (bude_pose_grad, bude_refine) takes at
 * most 8 poses per thread (FP64: 4) and, when its block comes from the
 * defaults, at most as many threads as the adjoint kernel's registers let
 * one CTA hold.  An explicit block that cannot be resident returns
 * BUDE_ERR_UNSUPPORTED.
 */
typedef struct {
    int32_t variant;     /* BUDE_FP32_IEEE .. BUDE_FP64 */
    int32_t ppwi;        /* poses per thread: 1, 2, 4, 8 or 16 (FP64: 1, 2, 4) */
    int32_t block;       /* threads per CTA: multiple of 32 in [64, 1024] */
    int32_t tile;        /* protein atoms staged per shared-memory chunk */
    int32_t ctas_per_sm; /* resident CTAs per SM of the persistent grid */
    int32_t cull;        /* 1: cutoff culling in the energy kernels (below); 0: default */
} bude_options;

/*
 * Cutoff culling (bude_options.cull = 1; no paper counterpart, off by
 * default).  Every term of the pair energy is exactly zero once d reaches
 * R + max(D_E, D_D) = R + 4 A.  With culling on, a warp computes the squared
 * distances of all its poses to a protein atom first and, when every one of
 * them lies beyond that cutoff (with a margin for the roots' rounding), skips
 * the roots and the terms for that atom.  The skipped terms would have added
 * exact zeros, so the energies are bit-identical to the unculled kernel of
 * the same launch shape; so are the pose gradients, whose terms and
 * derivatives vanish there too.  Built for the FP32 kernels with an even ppwi
 * (bude_energies, bude_energies_batched, bude_energies_noalloc,
 * bude_pose_grad, bude_refine); FP64, odd ppwi and bude_param_grad ignore the
 * flag.  Culled launches evaluate fewer pairs than Eq. 3 counts, so their
 * FLOP rate is not comparable with Eq. 3.
 */

typedef struct bude_deck bude_deck;

/*
 * bude_create_deck -- validate and repack one deck into buffers it owns.
 *
 * Copies desc's device arrays into the deck (the caller may free its own
 * copies once this call returns), maps each ligand type to a compact row of
 * the type-pair table and builds the pair parameters of the forcefield's
 * combination rules on the device (the table lookup of Eq. 3's 10 per-pair
 * FLOPs).  Runs on "stream" and SYNCHRONISES it to read the validation word.
 * Errors: BUDE_ERR_INVALID_ARG for null pointers, negative sizes,
 * n_types outside 1..BUDE_MAX_TYPES, an atom type outside [0, n_types), a
 * non-finite coordinate, a radius <= 0 or non-finite forcefield value, or an
 * hbtype outside {0, 1, 2}; BUDE_ERR_UNSUPPORTED when the pair table cannot
 * fit in shared memory; BUDE_ERR_OOM / BUDE_ERR_CUDA otherwise.  On error
 * *out is set to NULL.
 */
BUDE_API int bude_create_deck(const bude_deck_desc* desc, void* stream, bude_deck** out);

/* Free a deck and its workspace (synchronises the device first). NULL is OK. */
BUDE_API int bude_destroy_deck(bude_deck* deck);

/* Sizes recorded in a deck (any pointer may be NULL). */
BUDE_API int bude_deck_info(const bude_deck* deck, int32_t* n_lig, int32_t* n_pro,
                   int32_t* n_types, int32_t* n_rows);

/*
 * bude_energies -- energy of n poses (Listing 4, whole kernel).
 *
 * poses:    device float32 [6][n]: rows 0..2 are the angles about x, y, z,
 *           rows 3..5 the translation; the pose rotation is
 *           R = Rz(a2) Ry(a1) Rx(a0) (first element cos(a1) cos(a2) as in
 *           Listing 4) applied about the ligand's coordinate origin.
 * energies: device float32 [n], written as 0.5 * sum of pair energies.
 * opts:     NULL for defaults.
 * n = 0 is a no-op.  A deck with no ligand or no protein atoms yields zeros.
 * A pose whose transform has a NaN yields NaN.  The first call with a larger
 * n than before grows the deck's workspace: it synchronises "stream" when it
 * replaces a smaller workspace and allocates with cudaMalloc, so make such a
 * call before capturing the stream into a CUDA graph.
 */
BUDE_API int bude_energies(bude_deck* deck, const float* poses, int64_t n,
                  float* energies, const bude_options* opts, void* stream);

/*
 * bude_energies_host -- bude_energies with HOST poses and energies (the
 * end-to-end call; no paper counterpart).
 *
 * poses:    host float32 [6][n] (pinned memory lets the copies overlap).
 * energies: host float32 [n].
 * The call copies the poses into a device staging buffer the deck owns,
 * runs bude_energies on it and copies the energies back, all enqueued on
 * "stream"; the energies are in host memory once the stream has been
 * synchronised.  The first call with a larger n than before grows the
 * staging buffer (synchronising "stream" when it replaces a smaller one).
 * Same errors as bude_energies.  Calls on one deck must not overlap.
 */
BUDE_API int bude_energies_host(bude_deck* deck, const float* poses, int64_t n,
                                float* energies, const bude_options* opts, void* stream);

/*
 * bude_energies_batched -- many decks in one persistent launch.
 *
 * decks[i], poses[i] (device [6][n[i]]) and energies[i] (device [n[i]]) for
 * i < count describe independent docking problems of uneven sizes.  All of
 * them run in one launch of a persistent kernel that splits the combined
 * (pose tile x ligand atom x protein atom) space over the grid, evenly by
 * estimated cost (pairs with a desolvation term cost more).  The grid is
 * capped so that every CTA's share holds at least one unit.  The first call
 * with a given set of arguments builds a plan (work-list descriptors,
 * workspace) and captures the launch into a CUDA graph; calls with the same
 * arguments replay that graph.  The library keeps the 64 most recently used
 * plans; a plan dropped to make room is rebuilt by its next call, and its
 * destruction waits for the device.  Results equal bude_energies' within the
 * variant's rounding (the summation order differs).
 */
BUDE_API int bude_energies_batched(bude_deck* const* decks, const float* const* poses,
                          const int64_t* n, float* const* energies,
                          int32_t count, const bude_options* opts, void* stream);

/*
 * bude_energies_noalloc -- bude_energies for callers that must not allocate
 * device memory.  (The paper has no counterpart: this is a deployment
 * variant.)
 *
 * Some hosts own the whole device-memory budget and forbid allocation inside
 * their execution callbacks (plugins of inference servers and of other
 * frameworks with their own allocators), and latency-critical loops cannot
 * afford cudaMalloc's implicit synchronisation.  This call runs the same
 * kernel as bude_energies but keeps the kernel's scratch (cross-CTA partial
 * sums and arrival tickets) in one fixed array that the library declares in
 * device memory: 4 MiB of partial sums plus 64 KiB of tickets, held by every
 * GPU that loads the library until the process exits.  It calls no
 * cudaMalloc or cudaFree and no allocating routine; it clears the tickets
 * with cudaMemsetAsync and launches on "stream".
 *
 * Limits: a call needs (CTAs of the grid + pose tiles) x 32 x ppwi partial
 * sums and one ticket per pose tile of 32 x ppwi poses; with the tuned
 * shapes that is a few hundred thousand poses per call.  Larger calls return
 * BUDE_ERR_UNSUPPORTED with the sizes in bude_last_error().
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call shares the one array, so calls whose kernels overlap
 * on the GPU (different streams, or different threads) race and must be
 * serialised by the caller.  The looked-up address is kept for the life of
 * the process, so resetting or destroying a device's primary context
 * (cudaDeviceReset) while the library is loaded is not supported: later
 * calls on that device would use a stale address.  Arguments and results are
 * as bude_energies.
 */
BUDE_API int bude_energies_noalloc(bude_deck* deck, const float* poses, int64_t n,
                                   float* energies, const bude_options* opts, void* stream);

/*
 * bude_pose_grad -- energies and their gradient with respect to the six pose
 * parameters (the adjoint of bude_energies).
 *
 * grad: device float32 [6][n], d energy / d pose row j.  energies may be
 * NULL.  Variants BUDE_FP32_IEEE and BUDE_FP32_FAST (COMP maps to IEEE with
 * FP64 folds; FP64 computes in double).  A pair at zero distance adds no
 * gradient.
 */
BUDE_API int bude_pose_grad(bude_deck* deck, const float* poses, int64_t n,
                   float* energies, float* grad, const bude_options* opts,
                   void* stream);

/*
 * bude_selfcheck_sqrt -- diagnostics for the BUDE_FP32_IEEE energy kernels,
 * whose square root is computed without branches (Markstein's FMA
 * correction of an approximate reciprocal root).  Compares it bit for bit
 * with the correctly rounded sqrt over every float in [2^-100, 2^128) (the
 * kernels add 2^-100 to each squared distance) and stores the
 * number of mismatches (0 expected) and the smallest mismatching bit pattern
 * (0xffffffff when none).  Synchronises "stream".
 */
BUDE_API int bude_selfcheck_sqrt(uint64_t* mismatches, uint32_t* first_bad, void* stream);

/*
 * bude_refine -- on-device pose refinement (the docking step that follows
 * scoring; the paper's Sec. 2.2 describes docking but benchmarks only the
 * energy).  Per pose, "steps" iterations of normalised gradient descent with
 * an adaptive step:
 *   start:  E, g = energy and pose gradient at p;  alpha = step0
 *   step:   p' = p - alpha g / |g|   (p' = p when |g| is 0 or not finite)
 *           E', g' at p' (the adjoint kernel)
 *           if E' < E: p, E, g = p', E', g' and alpha *= 1.25, else alpha *= 0.5
 * so no pose's energy ever increases.  poses (device float32 [6][n]) is
 * updated in place; energies (device float32 [n]) receives the final E.
 * step0 is in pose units (radians and Angstrom share one step length).
 * The first call with a given argument set allocates the plan's buffers
 * (22 floats per pose, and its own partial-sum workspace, so that later calls
 * on the deck that resize the deck's workspace leave the graph valid) and
 * captures the whole loop -- 2 + 3 x steps kernel launches -- into one CUDA
 * graph; later calls replay it.  The 64 most recently used plans are kept, as
 * for bude_energies_batched.  Calls with one argument set must not overlap.
 * Variants and options as bude_pose_grad.
 */
BUDE_API int bude_refine(bude_deck* deck, float* poses, int64_t n, int32_t steps, float step0,
                         float* energies, const bude_options* opts, void* stream);

/*
 * bude_param_grad -- gradient of a weighted sum of pose energies,
 * L = sum_k w_k E_k, with respect to the ligand atom coordinates (in the
 * ligand's own frame, before the pose) and the per-type forcefield
 * parameters radius, hardness and elsc: the quantities forcefield fitting and
 * ligand design take from a scoring function.  (The paper benchmarks the
 * energy only; this differentiates it with respect to its other inputs.)
 *
 * weights:  device float32 [n], or NULL for all ones.
 * lig_grad: device float32 [n_lig][3], dL/d(x, y, z) per ligand atom.
 * ff_grad:  device float32 [n_types][3], dL/d(radius, hardness, elsc).
 * The hbtype class is discrete and has no gradient.  Variants BUDE_FP32_IEEE
 * and BUDE_FP32_FAST (COMP runs as IEEE); FP64 returns BUDE_ERR_UNSUPPORTED.
 * Sums are accumulated in FP64 in shared memory and added over CTAs in a
 * fixed order; shared-memory atomics make the last FP64 bits depend on
 * scheduling, which the float32 outputs do not see.  Uses the deck's
 * workspace: calls on one deck must not overlap.
 */
BUDE_API int bude_param_grad(bude_deck* deck, const float* poses, int64_t n,
                             const float* weights, float* lig_grad, float* ff_grad,
                             const bude_options* opts, void* stream);

/*
 * The paper's memory-bound kernels, kept as HBM calibration for this GPU
 * (Sec. 2.2, Listings 2 and 3; bandwidth metrics Eq. 1 and Eq. 2).
 *
 * bude_stream -- one BabelStream operation on n elements of device arrays
 * (dtype 0 float32, 1 float64; every array 16-byte aligned):
 *   op 0 copy  c = a        op 1 mul  b = scalar c      op 2 add  c = a + b
 *   op 3 triad a = b + scalar c                          op 4 dot  *dot_result = sum a b
 * dot_result is a device double (op 4 only), accumulated in FP64 and reduced
 * over CTAs in a fixed order through a fixed device array shared by all calls
 * (dot calls must not overlap on the GPU).  Asynchronous on "stream".
 */
BUDE_API int bude_stream(int32_t op, int32_t dtype, void* a, void* b, void* c, double scalar,
                         int64_t n, double* dot_result, void* stream);

/*
 * bude_laplacian -- seven-point stencil on an nx x ny x nz grid (Sec. 2.2,
 * Listing 2; bytes by Eq. 1), index i*ny*nz + j*nz + k, k fastest, interior
 * points only:
 *   f[i,j,k] = u[i,j,k] invhxyz2 + (u[i-1,j,k] + u[i+1,j,k]) invhx2
 *            + (u[i,j-1,k] + u[i,j+1,k]) invhy2 + (u[i,j,k-1] + u[i,j,k+1]) invhz2
 * Boundary points of f are not written.  u and f are distinct device arrays
 * of dtype 0 float32 or 1 float64.  Grids with a side below 3 are a no-op.
 * Both kernels evaluate the same expression in the same order, so the result
 * does not depend on which one runs.  BUDE_ERR_UNSUPPORTED: a grid beyond
 * the launch limits (ny or nx above about 2.6e5).  Asynchronous on "stream".
 *
 * bude_laplacian_path -- which kernel bude_laplacian takes for these
 * arguments (host logic only; u is not dereferenced): 1 the TMA kernel
 * (float32, u 16-byte aligned, nz a multiple of 4), 0 the register kernel,
 * or a negative error code for invalid arguments.
 *
 * bude_wait_timeouts -- synchronises "stream", then returns in *count, and
 * clears, the number of CTAs of the TMA stencil whose bounded wait for a
 * staged plane gave up (about a second) since the last call.  Such a CTA
 * leaves its tile of f unwritten for the rest of its planes, lets its copies
 * in flight land, and exits; the CUDA context stays usable.  0 in normal
 * operation.
 *
 * bude_debug_stall_next_stencil -- test hook: the next launch of the TMA
 * stencil has its first CTA skip the copy of its second computed plane, with
 * a wait limit of about a millisecond, so that exactly that CTA times out.
 */
BUDE_API int bude_laplacian(int32_t dtype, const void* u, void* f, int32_t nx, int32_t ny,
                            int32_t nz, double invhx2, double invhy2, double invhz2,
                            double invhxyz2, void* stream);
BUDE_API int bude_laplacian_path(int32_t dtype, const void* u, int32_t nx, int32_t ny, int32_t nz);
BUDE_API int bude_wait_timeouts(uint32_t* count, void* stream);
BUDE_API int bude_debug_stall_next_stencil(void);

/*
 * Hartree-Fock two-electron Fock term over s-type Gaussians (the paper's
 * other compute-bound kernel: Sec. 2.2, Listing 5, Table 4).  Every atom
 * carries one s function contracted from ngauss normalised primitives
 * (exponents xpnt, coefficients coef, the same on every atom); geometry in
 * bohr.  For a symmetric density D the call computes
 *   G_ij = sum_kl D_kl [ 2 (ij|kl) - (ik|jl) ]
 * from the unique integrals (i >= j, k >= l, ij >= kl) with the six Fock
 * updates of Listing 5 (FP64 atomics) and G = F + F^T.  Quartets whose
 * Schwarz bound sqrt((ij|ij) (kl|kl)) is below schwarz_tol are skipped.
 *
 * bude_hf_create: geom [n_atoms][3], xpnt and coef [ngauss] are HOST arrays
 *   (ngauss 1..8); builds the pair products and Schwarz bounds on the GPU and
 *   synchronises "stream".
 * bude_hf_fock: dens and g are device float64 [n][n] (row-major).  variant
 *   BUDE_FP64 evaluates every integral in FP64; BUDE_FP32_IEEE evaluates the
 *   primitive integrals in FP32 (GB300's FP64 rate is a small fraction of its
 *   FP32 rate) and accumulates in FP64.  Calls on one plan must not overlap.
 */
typedef struct bude_hf bude_hf;
BUDE_API int bude_hf_create(int32_t n_atoms, const double* geom, int32_t ngauss,
                            const double* xpnt, const double* coef, void* stream, bude_hf** out);
BUDE_API int bude_hf_fock(bude_hf* plan, const double* dens, double* g, double schwarz_tol,
                          int32_t variant, void* stream);
BUDE_API int bude_hf_destroy(bude_hf* plan);
/*
 * bude_hf_quartets: the number of unique quartets that survive schwarz_tol,
 * i.e. how many integrals (each of ngauss^4 primitive quartets) a
 * bude_hf_fock call with that threshold evaluates.  Synchronises "stream".
 */
BUDE_API int bude_hf_quartets(bude_hf* plan, double schwarz_tol, int64_t* count, void* stream);

/* Default options the library uses for a variant when a field is zero. */
BUDE_API int bude_get_default_options(int32_t variant, bude_options* out);
BUDE_API int bude_set_default_options(const bude_options* opts);

/* Kernel launches the last compute call on this thread enqueued. */
BUDE_API int64_t bude_last_launch_count(void);

BUDE_API const char* bude_status_string(int status);
BUDE_API const char* bude_last_error(void);

/*
 * Host-side fault injection for tests (no paper counterpart).  After
 * bude_debug_fail_alloc(n) with n > 0, the n-th device allocation the library
 * makes from then on fails as if the device were out of memory: the call that
 * makes it returns BUDE_ERR_OOM and must release whatever it had taken.  The
 * injection is one-shot and process-wide; n = 0 disarms it, n < 0 returns
 * BUDE_ERR_INVALID_ARG.  Nothing is allocated, freed or launched and no CUDA
 * call is made for the injected failure, so the CUDA context stays healthy.
 * bude_debug_pending_fail_alloc() returns how many allocations remain before
 * the injected failure (0 when disarmed): a call that allocates nothing leaves
 * it unchanged.
 */
BUDE_API int bude_debug_fail_alloc(int32_t n);
BUDE_API int32_t bude_debug_pending_fail_alloc(void);

/*
 * bude_debug_partition -- test hook: how the persistent kernel would split a
 * launch over its CTAs, computed on the host by the functions the kernel and
 * the planner use (no CUDA call; no paper counterpart).
 *
 * The launch has count instances; instance i has nt[i] pose tiles of K[i]
 * units each (K = ligand atoms x protein atoms), each unit costing w[i]
 * (launches of several instances weight a unit 100 + 40 x its deck's share
 * of pairs with a desolvation term, and split the total cost evenly).
 * grid: the CTAs the device could hold.  Outputs: *grid_out, the CTAs the
 * launch uses; and, each optional (NULL skips it):
 *   cta_begin[0 .. grid_out]: flat index where each CTA's range starts, the
 *               last entry one past the end;
 *   owner[N]:   the CTA whose range holds each flat unit, N = sum nt[i] K[i];
 *   cover[T]:   how many CTAs the kernel expects to finish each tile,
 *               T = sum nt[i].
 * Errors: BUDE_ERR_INVALID_ARG for count < 1, grid < 1, an empty instance or
 * a NULL size array.
 */
BUDE_API int bude_debug_partition(int32_t count, const int64_t* K, const int64_t* nt,
                                  const int32_t* w, int32_t grid, int32_t* grid_out,
                                  int64_t* cta_begin, int64_t* owner, int32_t* cover);

/*
 * bude_debug_cached_plans -- test hook: how many captured plans the library
 * holds for bude_energies_batched (*batched) and bude_refine (*refine); each
 * cache keeps at most 64 and drops the least recently used one when a call
 * with a new argument set needs room.  Either pointer may be NULL.  No CUDA
 * call.
 */
BUDE_API int bude_debug_cached_plans(int32_t* batched, int32_t* refine);

#ifdef __cplusplus
}
#endif
#endif /* BUDE_H */
