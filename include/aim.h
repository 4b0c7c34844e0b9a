/*
 * aim.h -- C ABI of the GB300 ET-AIM library (envelope-tracking adaptive integral
 * method for the time-domain EFIE on PEC surfaces).
 *
 * The library marches the complex current envelopes of Eq. 5,
 *
 *   (Z~near_0 + Z~FFT_0) I_l = V_l - sum_{m=1..N_g} (Z~near_m + Z~FFT_m) I_{l-m},
 *
 * with Z~FFT_m = anterpolation -> 3-D FFT convolution with the delayed grid
 * Green-function envelope -> interpolation (Sec. 4, stages i-iii), Z~near_m the
 * pre-corrected near-zone matrices (stage iv) and a diagonally preconditioned GMRES
 * for the immediate system (stage v; Sec. 5.1).  Unknowns are RWG current-envelope
 * coefficients (Eq. 3) for a CPPIF temporal basis.
 *
 * Conventions
 *  - Every call returns an int status (AIM_OK = 0, negative = error).  No C++
 *    exception crosses the ABI.  aim_last_error() returns a message for the last
 *    failing call on a context.
 *  - Complex numbers are interleaved (re, im) doubles: aim_c128.
 *  - Array arguments marked "host or device" may be either; the library
 *    classifies the pointer with cudaPointerGetAttributes and copies host
 *    arrays through internal staging buffers.  The caller owns every pointer it
 *    passes; the context owns all device memory it allocates.
 *  - A context is bound to one CUDA device and one stream (aim_opts.cuda_stream,
 *    or a stream it creates).  It is not thread-safe.
 *  - RWG ordering: interior edges sorted by (lower vertex, higher vertex); T+ is the
 *    face whose counter-clockwise cycle runs along the edge from the lower to the
 *    higher vertex.  aim_rwg_table() exports it.  Open surfaces (the plates of
 *    Sec. 5.1) are accepted: an edge of a single face is a boundary edge and carries
 *    no basis function.
 *  - Grid nodes are indexed n = (iz * N + iy) * N + ix; each RWG owns the 4x4x4
 *    stencil anchored at floor((x_e - origin)/h) - 1 (clamped to [0, N-4]) per
 *    axis, x_e the midpoint of its edge.
 */
#ifndef AIM_GB300_H
#define AIM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  AIM_OK = 0,
  AIM_ERR_ARG = -1,      /* invalid argument (null pointer, size out of range)     */
  AIM_ERR_MESH = -2,     /* non-manifold edge, inconsistent orientation, degenerate
                            face, or no interior edge                                 */
  AIM_ERR_CUDA = -3,     /* a CUDA runtime call failed (message in aim_last_error)  */
  AIM_ERR_OOM = -4,      /* device allocation failed                               */
  AIM_ERR_NOCONV = -5,   /* GMRES hit its iteration cap; stats->last_step is valid  */
  AIM_ERR_TIMEOUT = -6,  /* a bounded device wait gave up                           */
  AIM_WARN_UNSTABLE = 1  /* march finished, but the last |I_l| exceeds 1e3 x the
                            largest |I_l| of the first half of the run (late-time growth) */
};

enum { AIM_C128 = 0,     /* plain path: every stage in complex128                  */
       AIM_C64 = 1 };    /* grid stages (anterpolation, FFT, kernel multiply,
                            interpolation) in complex64 with FP32 accumulation;
                            near zone, residual and Krylov basis in FP64            */

enum { AIM_CPPIF = 0,    /* causal piecewise-polynomial interpolatory basis        */
       AIM_BLIF = 1 };   /* band-limited interpolatory basis (Sec. 3, 3.1.2): the
                            approximate prolate spheroidal interpolant
                            T(u) = sinc(u) w(u), |u| < M, w(u) = G(M^2 - u^2)/G(M^2),
                            G(s) = sinh(b sqrt s)/sqrt s, guard band
                            b = pi (1 - 2 aim_opts.blif_band); made causal by
                            extrapolating the samples l+1..l+M-1 from l..l-M+1
                            (least squares over 2M frequencies spread evenly over the
                            band, edges included), which folds them into Z_0..Z_{M-1} */

/* Right preconditioner of the immediate system (x = M y, solve Z_0 M y = b). */
enum { AIM_PRECOND_DIAG = 0,      /* M = diag(1 / Z_0[k,k]) (Sec. 5.1)                  */
       AIM_PRECOND_NEAR_SAI = 1 };/* no counterpart in the paper: M on the pattern of
                                     the RWG pairs within precond_radius (edge
                                     midpoints), column k minimising ||Zp[:, S_k] m - e_k||
                                     (S_k the pattern set of RWG k, Zp = Z_0 kept on the
                                     pattern).  A set wider than 144 RWGs is rejected.   */

typedef struct aim_ctx aim_ctx;                 /* opaque */
typedef struct { double re, im; } aim_c128;

typedef struct {
  int32_t nv, nt;
  const double* v;       /* [nv][3] vertex positions (m), host                      */
  const int32_t* tri;    /* [nt][3] vertex indices, counter-clockwise seen from
                            outside, host                                           */
} aim_mesh;

typedef struct {
  int32_t n;             /* nodes per axis (cubic grid N^3); x and y transforms of 2N
                            points, z transforms of aim_info.z_len points             */
  double origin[3];      /* position of node (0,0,0) (m)                            */
  double h;              /* node spacing (m)                                        */
} aim_grid;

typedef struct {
  int32_t kind;          /* AIM_CPPIF or AIM_BLIF                                   */
  int32_t order;         /* CPPIF: Q (1..4), support (-1, Q] in units of dt;
                            BLIF: the half-width M (2..5), support (-M, M); N_g is
                            floor(R_max / (c dt) + order) in both cases             */
} aim_tbasis;

typedef struct {
  double f_c;            /* carrier frequency (Hz); envelope x(t)=Re{x~ e^{j2pi f_c t}} */
  int32_t precision;     /* AIM_C128 or AIM_C64                                     */
  int32_t batch_max;     /* most right-hand sides marched together (>= 1)           */
  int32_t gmres_restart; /* Krylov dimension before restart (default 50 if <= 0)    */
  int32_t gmres_max_iter;/* iteration cap per step and RHS (default 500 if <= 0)    */
  void* cuda_stream;     /* cudaStream_t to run on, or NULL for a private stream    */
  int32_t preconditioner;/* AIM_PRECOND_DIAG (0, the paper's) or AIM_PRECOND_NEAR_SAI */
  double precond_radius; /* SAI pattern radius (m); <= 0: the near radius             */
  int32_t zero_start;    /* 0: GMRES starts from the previous step's currents (Sec. 5.1);
                            1: from zero, whose residual is b itself (no operator product
                            before the first Arnoldi step)                             */
  int32_t refine;        /* AIM_C64 only: FP64 refinement of every immediate solve.  0: off.
                            k > 0: after the complex64-operator GMRES, the residual
                            b - Z_0 x is formed with every grid stage in FP64; while its
                            relative norm exceeds tol, up to k correction solves
                            Z_0 d = r (complex64 operator, from zero, to 1e-2) update
                            x += d.  The march's tolerance then holds for the FP64
                            operator (AIM_ERR_NOCONV if k corrections do not reach it).  */
  int32_t refine_every;  /* with refine: check (and correct) the FP64 residual at every k-th
                            step only (k <= 1: every step); the other steps keep the complex64
                            solve                                                            */
  int32_t autotune;      /* launch shapes of the grid passes (the tile widths of the z and y
                            passes, rows per block of the x passes): 0 built-in defaults;
                            1 time every candidate on this context's buffers at setup and
                            keep the fastest, reusing a plan cached for the same GPU model,
                            padded lengths, precision and batch; 2 time and refresh the cache.
                            Cache: the file named by AIM_GB300_PLAN_CACHE, else
                            $HOME/.cache/aim_gb300_plans.jsonl (one JSON object per line).
                            The results do not depend on the plan (same arithmetic per line). */
  int32_t rhs_blocked;   /* 1: the march forms the delayed grid sums of Eq. 5 by the
                            multilevel blocked schedule of Sec. 4 stage ii: after step l
                            the z-spectra of its last b = 2^min(ctz(l), P) steps are
                            radiated at once to the next b steps' pending sums (2^P >= N_g),
                            so each step reads O(log N_g) spectra instead of N_g.  Needs a
                            power-of-two z transform (aim_info.z_len); holds 2^P source and
                            2^(P+1) pending z-spectra per right-hand side.  0: direct sums. */
  double eps_r, mu_r;    /* homogeneous background medium (Sec. 2.1): relative permittivity
                            and permeability; values <= 0 mean 1 (vacuum).  Light speed
                            c0 / sqrt(eps_r mu_r), mu = mu0 mu_r, eps = eps0 eps_r in every
                            kernel, excitation, far field and RCS.                          */
  double blif_band;      /* AIM_BLIF only: the envelope's half band times the time step,
                            f_bw dt, in (0, 1/2) (AIM_ERR_ARG otherwise).  With AIM_BLIF the
                            sampled-envelope excitation and far-field entry points
                            (aim_excitation_samples*, aim_farfield*, aim_march_farfield,
                            aim_march_adjoint_farfield) return AIM_ERR_ARG.                 */
} aim_opts;

typedef struct {
  int32_t nb;            /* number of plane waves (<= batch_max)                    */
  const double* khat;    /* [nb][3] unit propagation directions, host               */
  const double* phat;    /* [nb][3] unit polarisations, host                        */
  double sigma, t_d;     /* Gaussian width and delay of Eq. 1 (s)                   */
} aim_excitation;

typedef struct {
  int32_t last_step;     /* last completed step l (1-based)                         */
  int32_t total_iters;   /* GMRES iterations summed over steps and RHS              */
  int32_t max_iters;     /* largest per-step iteration count                        */
  double max_rel_res;    /* largest final relative residual over steps and RHS      */
  double rhs_ms;         /* device time in right-hand-side work (all steps)         */
  double solve_ms;       /* device time in the iterative solves (all steps, with the
                            FP64 refinement)                                          */
  int32_t* iters;        /* optional caller array [n_steps][nb] of iteration counts */
  int32_t refine_corrections; /* correction solves of the FP64 refinement (all steps)  */
  int32_t refine_checks; /* steps whose FP64 residual was formed (aim_opts.refine_every) */
} aim_stats;

typedef struct {
  int32_t ns;            /* RWG unknowns N_s                                        */
  int32_t n_delays;      /* N_g: largest delay with a non-zero grid kernel entry    */
  int32_t n_active;      /* grid nodes touched by some stencil                      */
  int64_t near_nnz;      /* near-zone pairs (one CSR pattern shared by all delays)  */
  int32_t grid_n;        /* N                                                       */
  int32_t precision;
  int64_t device_bytes;  /* device memory held by the context                       */
  int32_t preconditioner;/* AIM_PRECOND_*                                           */
  int64_t precond_nnz;   /* entries of the preconditioner's sparsity pattern          */
  int32_t refine;        /* aim_opts.refine as set up (0 on the complex128 path)       */
  int32_t refine_every;  /* aim_opts.refine_every as set up (>= 1)                       */
  int32_t plan_zw, plan_cw, plan_rp, plan_ypb; /* launch shapes in use (see aim_opts.autotune) */
  int32_t plan_source;   /* AIM_PLAN_*                                                  */
  int32_t box_lo[3], box_hi[3]; /* active box: grid nodes (x, y, z) touched by some stencil
                            lie in [box_lo, box_hi] (inclusive).  Sources vanish outside it
                            and potentials are needed only inside it, so every FFT pass but
                            the z pass (all lines, reading and writing only the box planes)
                            runs on the box's lines only, and the grid buffers hold the
                            box's z-planes only.                                          */
  int32_t rhs_blocked;   /* aim_opts.rhs_blocked as set up                                 */
  int32_t z_len;         /* length of the z transform: the shortest supported length
                            >= 2 (box_hi[2] - box_lo[2] + 1) (at most 2N).  The linear
                            convolution over the box's z-planes needs z offsets below the
                            box depth only, so this circular length gives the values of
                            the 2N padding on them.                                       */
} aim_info;

enum { AIM_PLAN_DEFAULT = 0, AIM_PLAN_MEASURED = 1, AIM_PLAN_CACHED = 2 };

/*
 * aim_setup -- build every table of the method on the device (Sec. 4 and Eq. 5):
 * RWG table, anterpolation coefficients by moment matching up to order 3 per
 * axis (Sec. 5.1), grid kernels G^A_m = (D^2 T)(m - R/c dt) e^{-j k_c R}/R and
 * G^phi_m = T(m - R/c dt) e^{-j k_c R}/R for m = 0..N_g (G(0) = 0) and their
 * zero-padded FFT spectra (2N x 2N x z_len: the z padding follows the depth of the
 * active box, aim_info), near-zone pairs (edge-midpoint distance <= near_radius;
 * negative: none), the Galerkin near-zone entries Z_m (FP64, singularity
 * extraction) minus their grid approximation, and the diagonal preconditioner.
 *   mesh, grid, opts: host structs;  dt: time step (s);  out: receives the context.
 * Errors: AIM_ERR_ARG, AIM_ERR_MESH, AIM_ERR_CUDA, AIM_ERR_OOM (nothing leaked).
 */
int aim_setup(const aim_mesh* mesh, const aim_grid* grid, double near_radius, double dt,
              aim_tbasis tbasis, const aim_opts* opts, aim_ctx** out);

/* Release every device allocation of the context.  Safe on NULL. */
void aim_destroy(aim_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failed aim_setup if ctx is NULL). */
const char* aim_last_error(const aim_ctx* ctx);

int aim_get_info(const aim_ctx* ctx, aim_info* info);

/* Kernels of the library, for aim_get_profile. */
enum {
  AIM_K_ANTERP_XFFT = 0, /* anterpolation gather + forward x-FFT                          */
  AIM_K_YFFT_FWD,        /* forward y-FFT (pruned input)                                   */
  AIM_K_ZCONV,           /* forward z-FFT, kernel product, inverse z-FFT (immediate term)  */
  AIM_K_ZRHS,            /* delay sum over the N_g z-spectra of the history, inverse z-FFT */
                         /* (forward z-FFTs per delay for lengths with a factor 3)        */
  AIM_K_YFFT_INV,        /* inverse y-FFT (pruned output)                                  */
  AIM_K_XFFT_INV,        /* inverse x-FFT (pruned output)                                  */
  AIM_K_INTERP_NEAR,     /* interpolation gather + near-zone CSR product                   */
  AIM_K_EXCITATION,      /* excitation vector V_l                                          */
  AIM_K_GMRES_DOT,       /* separate Krylov dot kernel (systems beyond 32 768 unknowns;    */
                         /* smaller ones form the dots in the interpolation kernel)       */
  AIM_K_GMRES_UPDATE,    /* Gram-Schmidt updates with their reductions and column finish,  */
                         /* residual norms                                                 */
  AIM_K_GMRES_SMALL,     /* cycle start, rotations + back substitution, solution update    */
  AIM_K_PREP,            /* operator input: selection, Krylov scale, preconditioner, cast  */
  AIM_K_ZFWD,            /* z-spectrum of a committed history slab (power-of-two lengths)  */
  AIM_K_BLOCK_SQUARE,    /* blocked right-hand side: one square of source/observer steps   */
  AIM_K_ZINV_PENDING,    /* blocked right-hand side: pending z-spectra -> potentials slab  */
  AIM_K_COUNT
};

/*
 * aim_profile -- reset the kernel counters; enable != 0 also records a CUDA event
 * pair around every kernel launch on the context stream (device time per kernel).
 * aim_get_profile -- launches[AIM_K_COUNT] and total device ms[AIM_K_COUNT] since
 * the last reset (ms only while profiling was enabled), and the total number of
 * kernel launches (always counted).  Host arrays; either may be NULL.
 * aim_kernel_name -- a static name for a kernel id ("?" if out of range).
 */
int aim_profile(aim_ctx* ctx, int32_t enable);
int aim_get_profile(aim_ctx* ctx, int64_t* launches, double* ms, int64_t* total_launches);
const char* aim_kernel_name(int32_t id);

/* N_s and N_g of the context. */
/* aim_time_factor -- the temporal basis on the host, no context or GPU needed (Sec. 3, Eq. 3
 * and Sec. 3.1.2): out[i][d] = d-th derivative (d = 0..3, in units of the step) of the time
 * factor of delay m at x[i] = R / (c dt), i = 0..n-1: T(m - x) for AIM_CPPIF; for AIM_BLIF
 * T(m - x) plus, for m < M, the extrapolated samples sum_p E[p][m] T(-p - x) (the factor the
 * context's Z_m is built with).  x and out are host arrays ([n], [n][4]), owned by the caller.
 * AIM_ERR_ARG for a bad basis, order or blif_band (aim_last_error(NULL) says which), m < 0,
 * n < 0 or null arrays. */
int aim_time_factor(aim_tbasis tbasis, double blif_band, int32_t m, int32_t n, const double* x, double* out);

int aim_num_unknowns(const aim_ctx* ctx, int32_t* ns, int32_t* n_delays);

/*
 * aim_rwg_table -- the RWG ordering used by every vector of the library.
 *   edge [ns][2] (lower, higher vertex), tri [ns][2] (T+, T-), free_vertex [ns][2]
 *   (vertex opposite the edge in T+, T-).  Host arrays supplied by the caller.
 */
int aim_rwg_table(const aim_ctx* ctx, int32_t* edge, int32_t* tri, int32_t* free_vertex);

/*
 * aim_matvec -- y = Z~AIM_m x = Z~FFT_m x + Z~near_m x (Eq. 5), for delay
 * 0 <= m <= N_g and nb <= batch_max right-hand sides.
 *   x, y: [nb][ns] aim_c128, host or device.  In AIM_C64 the grid part runs in
 *   complex64 and the near part in FP64; y is accumulated in FP64.
 */
int aim_matvec(aim_ctx* ctx, int32_t delay_m, int32_t nb, const aim_c128* x, aim_c128* y);

/*
 * aim_matvec_noalloc -- the same product as aim_matvec, for callers that must not
 * allocate device memory while they run: a real-time or certified path whose memory is
 * fixed at start-up, an application whose device memory belongs to another allocator
 * (a framework's caching pool it must not bypass), a process under a hard device-memory
 * quota.  The paper has no counterpart: this is a library convenience.
 *   Allocates nothing (no cudaMalloc/cudaFree, no allocating library call).  The
 *   grid work space comes from one fixed 16 MiB device array in the library, held by
 *   every GPU that loads it until process exit; the context's other tables are used
 *   as set up by aim_setup.  nb * 4 * nz * (N*2N + 2N*2N + N^2) elements (complex64 or
 *   complex128 by precision; nz = the active box's z-planes, aim_info.box_lo/box_hi)
 *   must fit in 16 MiB, else AIM_ERR_ARG (e.g. N <= 32 in complex64 for one
 *   right-hand side).  The first call on a device looks up the
 *   array's device address (cudaGetSymbolAddress) with that device current and keeps
 *   it for the process; the kept address does not survive cudaDeviceReset, so do not
 *   call this entry point on a device after resetting it.  All calls share the array,
 *   so calls whose work overlaps on the GPU (two streams, two contexts) race; nothing in
 *   it needs to start at zero, and it keeps the last call's contents.
 *   x, y: [nb][ns] aim_c128, host or device, not overlapping.  The call returns after
 *   synchronising the context's stream.
 */
int aim_matvec_noalloc(aim_ctx* ctx, int32_t delay_m, int32_t nb, const aim_c128* x, aim_c128* y);

/*
 * aim_rhs -- the delayed-interaction sum of Eq. 5 at step l:
 *   rhs = sum_{m=1..N_g, l-m >= 1} Z~AIM_m I_{l-m}.
 *   hist: [N_g][nb][ns] with hist[m-1] = I_{l-m} (entries with l - m < 1 are
 *   ignored); rhs: [nb][ns].  Host or device.  The grid part is one spectral-domain
 *   delay sum (one inverse transform for all delays).
 */
int aim_rhs(aim_ctx* ctx, int32_t step_l, int32_t nb, const aim_c128* hist, aim_c128* rhs);

/*
 * aim_excitation_vector -- V_l[k] = <S_k, D E~inc(., l dt)> for the modulated
 * Gaussian plane waves of Eq. 1 (D = d/dt + j w_c), Cowper 7-point cubature.
 *   out: [nb][ns], host or device.
 */
int aim_excitation_vector(aim_ctx* ctx, const aim_excitation* exc, int32_t step_l, aim_c128* out);

/*
 * aim_march -- solve Eq. 5 for l = 1..n_steps starting from rest (I_l = 0, l <= 0).
 * Each step: excitation, delayed sum (spectral history ring), then GMRES on the
 * immediate system to relative residual tol, warm-started from I_{l-1}.
 *   currents: [n_steps][nb][ns] aim_c128, host or device (written step by step).
 *   stats: optional.  Returns AIM_ERR_NOCONV if a solve hits gmres_max_iter, or the
 *   FP64 refinement (aim_opts.refine) does not reach tol at a checked step (steps up to
 *   stats->last_step are valid), AIM_WARN_UNSTABLE if the march completed with late-time
 *   growth.
 */
int aim_march(aim_ctx* ctx, const aim_excitation* exc, int32_t n_steps, double tol,
              aim_c128* currents, aim_stats* stats);

/*
 * aim_march_continue -- advance a march started by aim_march by n_steps more steps,
 * using the history held in the context (the last N_g currents and their grid
 * spectra).  exc must describe the same plane waves (same nb) as the aim_march
 * call that started it.  currents: [n_steps][nb][ns], host or device.  Returns
 * AIM_ERR_ARG if no march was started on this context.
 */
int aim_march_continue(aim_ctx* ctx, const aim_excitation* exc, int32_t n_steps, double tol,
                       aim_c128* currents, aim_stats* stats);

/*
 * Gradients (not in the paper: the linear maps around the march of Eq. 5, used to
 * differentiate a far-field objective with respect to the incident envelope).
 *
 * aim_march_source -- march Eq. 5 from rest with explicit right-hand sides S_l in
 * place of the plane-wave excitation: sum_m Z_m I_{l-m} = S_l (transpose = 0), or with
 * every Z_m replaced by its transpose Z_m^T (transpose = 1; the grid part is symmetric,
 * the near-zone values are transposed).  The adjoint march M^H lam = G is the
 * transposed march of conj(G) in reversed time, conjugated.
 *   src, currents: [n_steps][nb][ns], host or device.
 *
 * aim_excitation_samples -- V_l[k], l = 1..n_steps, for the incident envelope
 * e(tau) = sum_i a_i T(tau/dt - i) (the CPPIF interpolant of envelope samples
 * a_i, i = i0..i0+n_samp-1) of a plane wave (khat, phat: host [3]):
 *   V_l[k] = sum_i a_i <S_k, phat (DT)(l - i - r.khat/(c dt)) e^{-j k_c r.khat}>,
 *   (DT)(u) = T'(u)/dt + j w_c T(u)  (Eq. 1 and Eq. 4 with a sampled envelope).
 *   a: [n_samp], V: [n_steps][ns]; host or device.
 * aim_excitation_samples_adjoint -- its adjoint: grad_i = sum_l sum_k conj(B_{l-i}[k])
 *   lam_l[k] for lam [n_steps][ns] -> grad [n_samp].
 *
 * aim_farfield -- far-field envelope in nd directions rhat [nd][3] with transverse
 * unit vectors e1, e2 [nd][3] (host), n = n0..n0+n_out-1:
 *   F[n][d][q] = -mu/(4 pi) sum_l sum_k I_l[k] int S_k.e_q (DT)(n - l + rhat.r'/(c dt))
 *                e^{+j k_c rhat.r'} dS',   I: [n_steps][ns], F: [n_out][nd][2].
 * aim_farfield_adjoint -- G_l[k] = sum_n sum_{d,q} conj(coefficient of I_l[k] in
 *   F[n][d][q]) F[n][d][q] for the given F -> G [n_steps][ns] (= dJ/d conj(I) for
 *   J = sum |F|^2).
 * All cubatures use the 7-point rule; errors: AIM_ERR_ARG on null pointers or sizes.
 */
int aim_march_source(aim_ctx* ctx, int32_t transpose, int32_t nb, int32_t n_steps, const aim_c128* src,
                     double tol, aim_c128* currents, aim_stats* stats);

/*
 * aim_march_adjoint -- the adjoint march M^H lam = G of the march of Eq. 5 (M block
 * lower-triangular Toeplitz in Z_0..Z_{N_g}): lam_l solves
 *   Z_0^H lam_l = G_l - sum_{m=1..N_g, l+m <= n_steps} Z_m^H lam_{l+m},  l = n_steps..1,
 * run as the transposed march of conj(G) in reversed time, conjugated (Z_m^H =
 * conj(Z_m^T); the grid part is symmetric, the near-zone values are transposed).  Only
 * the N_g most recent adjoint states are held.
 *   G, lam: [n_steps][nb][ns], host or device.  stats and errors as aim_march.
 */
int aim_march_adjoint(aim_ctx* ctx, int32_t nb, int32_t n_steps, const aim_c128* G, double tol, aim_c128* lam,
                      aim_stats* stats);

/*
 * aim_march_farfield -- forward pass of the far-field objective without a current
 * history: march Eq. 5 from rest for the sampled-envelope excitation of one plane wave
 * (as aim_excitation_samples: samples a [n_samp], i = i0..) and add each committed I_l's
 * contribution to the far-field envelope F (as aim_farfield: nd directions, n = n0..
 * n0+n_out-1) as soon as it is committed.  Only the march's N_g-step history exists.
 *   F: [n_out][nd][2], host or device (overwritten).  stats and errors as aim_march.
 *
 * aim_march_adjoint_farfield -- its adjoint: grad = B^H M^{-H} A^H F, i.e. the
 * derivative dJ/d conj(a) of J = sum |F|^2 (B: samples -> excitation, A: currents -> far
 * field).  The adjoint march runs in reversed time; at each of its steps the source
 * G_l = A^H F is formed for that l only and lam_l is added into grad at once, so neither
 * G nor lam is ever stored for all steps.  F: [n_out][nd][2], grad: [n_samp]; host or
 * device.
 */
int aim_march_farfield(aim_ctx* ctx, const double* khat, const double* phat, int32_t i0, int32_t n_samp,
                       const aim_c128* a, int32_t n_steps, double tol, int32_t nd, const double* rhat,
                       const double* e1, const double* e2, int32_t n0, int32_t n_out, aim_c128* F,
                       aim_stats* stats);
int aim_march_adjoint_farfield(aim_ctx* ctx, const double* khat, const double* phat, int32_t i0, int32_t n_samp,
                               int32_t n_steps, double tol, int32_t nd, const double* rhat, const double* e1,
                               const double* e2, int32_t n0, int32_t n_out, const aim_c128* F, aim_c128* grad,
                               aim_stats* stats);

/*
 * aim_march_spectrum -- the frequency-domain currents of a march (Sec. 2.4): march Eq. 5
 * from rest for the plane waves of exc (as aim_march) and, instead of the current
 * history, return for each frequency f the current for a unit incident plane wave
 *   I_f[b][k] = dt That(Omega dt) sum_l I_l[b][k] e^{-j Omega l dt} / E~(Omega),
 *   Omega = 2 pi (f - f_c),  That(w) = int T(u) e^{-j w u} du  (the CPPIF of Eq. 3),
 *   E~(Omega) = sigma sqrt(2 pi) exp(-sigma^2 Omega^2 / 2) exp(-j (w_c + Omega) t_d),
 * E~ being the transform of the incident envelope of Eq. 1 at the origin (envelope
 * convention x(t) = Re{x~(t) e^{j w_c t}}).  Each committed I_l is added at once; no
 * current history is kept.  The march cannot be continued (aim_march_continue).
 *   freqs: host [n_freq] (Hz, > 0), 1 <= n_freq <= 64; spec: [n_freq][nb][ns], host or
 *   device.  stats and errors as aim_march.
 *
 * aim_rcs -- bistatic RCS (m^2) of frequency-domain currents for a unit incident field:
 *   sigma[f][b][d] = 4 pi (w mu0 / (4 pi))^2 |pol_d . (I - r_d r_d) sum_k I_f[b][k]
 *                    int S_k(r') e^{+j k r_d.r'} dS'|^2,   w = 2 pi f_f,  k = w / c
 * (the 7-point cubature of every face).  With the currents of aim_march_spectrum this
 * is the co- or cross-polarised RCS of the march at f, the quantity the dB-error norm
 * of Eq. 2 compares over all directions.
 *   freqs: host [n_freq]; spec: [n_freq][nb][ns] host or device; rhat, pol: host
 *   [nd][3] unit vectors; sigma: [n_freq][nb][nd] host or device.  AIM_ERR_ARG on null
 *   pointers or sizes outside 1..65535.
 */
int aim_march_spectrum(aim_ctx* ctx, const aim_excitation* exc, int32_t n_steps, double tol, int32_t n_freq,
                       const double* freqs, aim_c128* spec, aim_stats* stats);
int aim_rcs(aim_ctx* ctx, int32_t n_freq, const double* freqs, int32_t nb, const aim_c128* spec, int32_t nd,
            const double* rhat, const double* pol, double* sigma);

int aim_excitation_samples(aim_ctx* ctx, const double* khat, const double* phat, int32_t i0, int32_t n_samp,
                           const aim_c128* a, int32_t n_steps, aim_c128* V);
int aim_excitation_samples_adjoint(aim_ctx* ctx, const double* khat, const double* phat, int32_t i0,
                                   int32_t n_samp, int32_t n_steps, const aim_c128* lam, aim_c128* grad);
int aim_farfield(aim_ctx* ctx, int32_t nd, const double* rhat, const double* e1, const double* e2,
                 int32_t n_steps, const aim_c128* I, int32_t n0, int32_t n_out, aim_c128* F);
int aim_farfield_adjoint(aim_ctx* ctx, int32_t nd, const double* rhat, const double* e1, const double* e2,
                         int32_t n_steps, int32_t n0, int32_t n_out, const aim_c128* F, aim_c128* G);

/*
 * Parity access to the setup tables (host arrays supplied by the caller).
 *   aim_get_anterp: anchor [ns][3] (int32), lam [ns][4][64] (x, y, z, div rows;
 *     stencil node t = (dz*4 + dy)*4 + dx).
 *   aim_get_near: rowptr [ns+1], col [nnz], val [(N_g+1)][nnz] aim_c128 (the
 *     pre-corrected Z~near_m).
 *   aim_get_kernel_spectrum: the stored octant [z_len/2 + 1][N+1][N+1] (kz, ky, kx) of
 *     the spectrum of G^A_m (kind 0) or G^phi_m (kind 1) on the (2N, 2N, z_len) padded
 *     grid (offsets |d| < N in x and y, |dz| < z_len/2 in z, even-symmetric
 *     embedding), including the folded constants mu/(4 pi) or 1/(4 pi eps) and
 *     1/(4 N^2 z_len).
 *   aim_get_preconditioner: the right preconditioner M in CSR form: rowptr [ns+1],
 *     col [precond_nnz], val [precond_nnz] aim_c128 with val[e] = M[row, col[e]]
 *     (AIM_PRECOND_DIAG: one diagonal entry per row).
 */
int aim_get_anterp(const aim_ctx* ctx, int32_t* anchor, double* lam);
int aim_get_near(const aim_ctx* ctx, int32_t* rowptr, int32_t* col, aim_c128* val);
int aim_get_preconditioner(const aim_ctx* ctx, int32_t* rowptr, int32_t* col, aim_c128* val);
int aim_get_kernel_spectrum(const aim_ctx* ctx, int32_t delay_m, int32_t kind, aim_c128* out);

#ifdef __cplusplus
}
#endif

#endif /* AIM_GB300_H */
