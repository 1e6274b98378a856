/*
 * helm.h - C ABI of libhelm: batched 2D Helmholtz solves on one GB300
 * (sm_103a) for frequency-domain full waveform inversion.
 *
 * What is solved (Sec. 3.1, Eq. 3.1-3.2): for a medium kappa = 1/c (s/m,
 * squared slowness m = kappa^2) and an absorbing-layer profile gamma,
 *
 *     H(m, w) u = -Lap_h u - w^2 m (1 - i gamma) u = g
 *
 * with the second-order five-point Laplacian on a node grid of spacings
 * (hx, hz) and zero values on the ghost nodes outside the grid.  The solver
 * is restarted flexible GMRES preconditioned by a shifted-Laplacian multigrid
 * V-cycle (Sec. 3.4, Eq. 3.12) or by the encoder-solver network followed by
 * that V-cycle (M_VU, Eq. 3.14).  Adjoint systems H^* x = b are solved with
 * the same operator through conjugation (Sec. 4.3, Eq. 4.8).
 *
 * Layout.  Every field is row-major [nz][nx] (x fastest); a batch of fields
 * is [nrhs][nz][nx].  Complex values are interleaved (re, im).
 *
 * Pointers.  Array arguments may be device pointers or host pointers; the
 * library detects which (cudaPointerGetAttributes) and stages host data
 * through its own device buffers on the context's stream.  The caller keeps
 * ownership of every buffer it passes; the library owns the context, the
 * multigrid hierarchy and all Krylov workspace.
 *
 * Errors.  Every function returns an int status (HELM_OK = 0); nothing is
 * thrown across the ABI.  helm_last_error() returns a thread-local message
 * describing the most recent failure on the calling thread.
 *
 * Streams.  All device work of a context is issued on opts.stream (a
 * cudaStream_t, NULL for the legacy default stream).  helm_solve blocks the
 * host until the batch has converged (it reads per-RHS convergence flags
 * once per restart cycle).  A context must not be used from two host
 * threads at once.
 */
#ifndef HELM_H
#define HELM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } helm_c64;
typedef struct { double re, im; } helm_c128;

typedef struct helm_ctx helm_ctx;     /* opaque, library-owned */
typedef struct cnn_model cnn_model;   /* opaque, library-owned */

enum {
    HELM_OK = 0,
    HELM_EINVAL = 1,        /* bad argument: sizes, pointers, options          */
    HELM_ENOMEM = 2,        /* device or host allocation failed                */
    HELM_ECUDA = 3,         /* a CUDA runtime call failed                      */
    HELM_ENOCONV = 4,       /* some RHS missed tol within max_iter (others ok) */
    HELM_EBREAKDOWN = 5,    /* NaN/Inf appeared for some RHS                   */
    HELM_ETIMEOUT = 6,      /* a bounded device wait expired                   */
    HELM_EUNSUPPORTED = 7   /* option combination not implemented              */
};

enum { HELM_PC_NONE = 0, HELM_PC_MG = 1, HELM_PC_CNN = 2 };
enum { HELM_COARSE_GMRES = 0, HELM_COARSE_JACOBI = 1 };
enum { HELM_OP_H = 0, HELM_OP_SL = 1 };
enum { HELM_SOLVE_ADJOINT = 1, HELM_SOLVE_ZERO_X0 = 2 };   /* helm_solve flags */

/* Solver options.  helm_default_opts() fills the defaults shown. */
typedef struct {
    int   restart;          /* FGMRES restart length k                     (10)  */
    int   max_iter;         /* total FGMRES steps per RHS (Sec. 5.7 cap)  (300)  */
    int   mg_levels;        /* V-cycle levels, >= 2                          (3)  */
    int   pre, post;        /* damped-Jacobi sweeps before / after          (2,2) */
    float jacobi_w;         /* Jacobi damping                              (0.8)  */
    float sl_beta;          /* shift beta of Eq. 3.12, alpha = 1           (0.5)  */
    int   sl_include_gamma; /* 1: shift w^2 m (1 - i(beta+gamma)); 0: Eq. 3.12 literal (1) */
    int   coarse_kind;      /* HELM_COARSE_GMRES or HELM_COARSE_JACOBI           */
    int   coarse_iters;     /* steps of the coarsest-level solve            (10)  */
    int   precond;          /* HELM_PC_MG, HELM_PC_CNN or HELM_PC_NONE          */
    int   max_rhs;          /* RHS per device batch; larger calls are chunked (256) */
    int   cnn_vcycle;       /* M_VU composition (Eq. 3.14): 0 = e_0 + V(r - H e_0); 3 = a e_0 + V(r - a H e_0)
                               with a = 1 unless ||r - H e_0|| > ||r||, then the complex a minimising
                               ||r - a H e_0||; 2 = 0 for every RHS until one of its restart cycles
                               lowers the residual by less than 10 %, then 3 for that RHS; 1 = V-cycle
                               on P u = r from u_0 = e_0                                      (2) */
    int   autotune;         /* 1: helm_setup runs helm_autotune (sweeps, and convolutions with a network)
                               on max_rhs RHS                                                 (0) */
    void* stream;           /* cudaStream_t for all work of the context   (NULL) */
} helm_opts;

/* Per-RHS results of helm_solve, caller-allocated HOST arrays of nrhs entries
 * (any pointer may be NULL). */
typedef struct {
    int*    iters;          /* FGMRES steps taken                              */
    double* rel_res;        /* final ||b - H x||_2 / ||b||_2, evaluated in FP64 */
    int*    status;         /* HELM_OK, HELM_ENOCONV or HELM_EBREAKDOWN         */
} helm_stats;

void helm_default_opts(helm_opts* opts);

/* Create a context for one medium and a set of angular frequencies.
 *   kappa, gamma : float32 [nz][nx] (kappa = 1/c in s/m; gamma >= 0 absorbing layer)
 *   omegas       : float32 [nfreq], angular frequencies w = 2 pi f (rad/s), host or device
 *   hx, hz       : grid spacings (m)
 *   net          : encoder-solver network for HELM_PC_CNN (its encoder runs here, once per
 *                  frequency, Eq. 3.13); NULL for the multigrid preconditioner
 * nx and nz must be divisible by 2^(mg_levels-1).  Builds the Galerkin multigrid
 * hierarchy of the shifted Laplacian for every frequency (Sec. 3.4) on the device.
 * Returns HELM_EINVAL on bad sizes/options, HELM_ENOMEM if the workspace for
 * opts.max_rhs right-hand sides does not fit. */
int helm_setup(helm_ctx** out, const float* kappa, const float* gamma, int nx, int nz,
               float hx, float hz, const float* omegas, int nfreq,
               const cnn_model* net, const helm_opts* opts);

/* Replace the medium (and the frequencies, same count) of an existing context and
 * rebuild its multigrid hierarchy on the device: the per-medium set-up of Sec. 3.4
 * without reallocating the workspace (FWI changes the medium every iteration). */
int helm_set_medium(helm_ctx* ctx, const float* kappa, const float* gamma,
                    const float* omegas, int nfreq);

/* Solve H(m, w_f) x = rhs, or H^* x = rhs with flags & HELM_SOLVE_ADJOINT (Eq. 4.8)
 * for nrhs right-hand sides, to ||b - H x||_2 <= tol ||b||_2 with the residual
 * evaluated in FP64 from the FP64 iterate.
 *   rhs      : complex64 [nrhs][nz][nx]
 *   x        : complex128 [nrhs][nz][nx]; in: initial guess (not read when
 *              flags & HELM_SOLVE_ZERO_X0: the guess is then zero); out: solution.
 *              The iterate is kept in complex128 because the complex64 rounding
 *              of a point-source solution alone leaves a relative residual near 1e-6.
 *   freq_idx : host int32 [nrhs], index into the context's omegas per RHS (NULL: all 0)
 * Returns HELM_OK when every RHS converged, HELM_ENOCONV / HELM_EBREAKDOWN when some
 * did not (see stats), or an error code. */
int helm_solve(helm_ctx* ctx, const helm_c64* rhs, helm_c128* x, int nrhs,
               const int* freq_idx, double tol, int flags, helm_stats* stats);

/* r = rhs - H(m, w_f) x evaluated in FP64 from the complex128 x (the check that
 * decides convergence in helm_solve), stored as complex64, and the per-RHS relative
 * residual ||r||_2 / ||rhs||_2 (FP64) into the host array rel_res (may be NULL). */
int helm_residual(helm_ctx* ctx, const helm_c64* rhs, const helm_c128* x, helm_c64* r, int nrhs,
                  const int* freq_idx, double* rel_res);

/* helm_residual_noalloc: the same FP64 residual and relative norms as helm_residual,
 * for callers that cannot allocate device memory - a process whose device memory is
 * reserved by another allocator (a framework's caching pool that owns the budget), or a
 * latency-critical loop where an allocation, and the synchronisation it can imply, is not
 * acceptable.  The paper has no counterpart; this is a deployment convenience.
 * It allocates nothing and needs no context: every array is a caller-owned DEVICE
 * pointer of the current device (a host pointer, or memory of another GPU, is rejected
 * with HELM_EINVAL; managed memory is accepted), the work is issued on `stream`
 * (a cudaStream_t, NULL = legacy default stream) and the call returns without waiting.
 *   kappa, gamma : float32 [nz][nx];  omega_rhs : float32 [nrhs], w of each RHS (rad/s)
 *   rhs : complex64 [nrhs][nz][nx];  x : complex128 [nrhs][nz][nx]
 *   r (out) : complex64 [nrhs][nz][nx] = rhs - H x;  rel_res (out) : double [nrhs] on device
 * Scratch: a fixed 1 MiB + 16 KiB file-scope device array that every GPU loading the
 * library holds until exit; a call needs nrhs <= 4096 and nrhs * ceil(nx/32) *
 * ceil(nz/64) <= 65536 (1024 right-hand sides of 512 x 256), larger sizes return
 * HELM_EINVAL with the limits in helm_last_error().  Every call shares that array and
 * clears its counters on `stream` first, so calls that overlap on the GPU (different
 * streams, or different host threads) race and must be serialised by the caller.
 * The first call on each device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture. */
int helm_residual_noalloc(const float* kappa, const float* gamma, int nx, int nz, float hx, float hz,
                          const float* omega_rhs, const helm_c64* rhs, const helm_c128* x, helm_c64* r,
                          double* rel_res, int nrhs, void* stream);

/* y = A x for A = H(m, w_f) (op = HELM_OP_H, Eq. 3.2) or the fine shifted Laplacian
 * P (op = HELM_OP_SL, Eq. 3.12 with the context's shift options); complex64 in/out. */
int helm_apply(helm_ctx* ctx, const helm_c64* x, helm_c64* y, int nrhs,
               const int* freq_idx, int op);

/* u = V-cycle(P, f, u0): one multigrid cycle of the context's hierarchy on P u = f
 * from the initial guess u0 (NULL: zero), Sec. 3.4 / Eq. 3.14.  complex64. */
int helm_vcycle(helm_ctx* ctx, const helm_c64* f, const helm_c64* u0, helm_c64* u,
                int nrhs, const int* freq_idx);

/* FWI data misfit and its gradient with respect to the squared slowness m = kappa^2
 * (Eq. 3.5 with Sigma = I and no regulariser; adjoint-state gradient, Sec. 4.3):
 *     Phi = sum_{j,s} || P^T u_sj - d_sj ||^2,   u_sj = H(m, w_j)^{-1} e_{src_s} / (hx hz)
 *     dPhi/dm = sum_{j,s} 2 w_j^2 Re((1 - i gamma) u_sj mu_sj),  mu_sj = H^{-1} P conj(P^T u_sj - d_sj)
 * for every frequency j of the context and every source s.  The adjoint field mu is the
 * conjugate of the solution of H^* lambda = P r (Eq. 4.8), obtained with a forward solve.
 *   src_idx : host int32 [nsrc], flat grid index iz * nx + ix of each point source
 *   rcv_idx : host int32 [nrcv], flat grid index of each receiver (all sources share them)
 *   d_obs   : complex64 [nfreq][nsrc][nrcv] observed data (host or device)
 *   tol     : relative residual of the forward and adjoint solves
 *   misfit_out : host double;  grad_m_out : float32 [nz][nx] (host or device)
 * The nfreq x nsrc (frequency, source) pairs are solved in chunks of up to max_rhs pairs
 * (a frequency's sources may span two chunks).  Allocates its forward/adjoint wavefields
 * per call (2 x 16 bytes per grid point and pair of one chunk).  Returns the first failing
 * helm_solve status, or HELM_OK. */
int fwi_misfit_grad(helm_ctx* ctx, const int* src_idx, int nsrc, const int* rcv_idx, int nrcv,
                    const helm_c64* d_obs, double tol, double* misfit_out, float* grad_m_out);

/* ---- Gauss-Newton FWI (Sec. 3.2-3.3, Alg. 1) ------------------------------------------
 * A survey: point-source nodes src_idx[nsrc] and receiver nodes rcv_idx[nrcv] (flat grid
 * indices iz * nx + ix, host int32; every source shares the receivers).  With src_w ==
 * NULL the sources are the nsrc point sources e_s / (hx hz); otherwise there are nsim
 * simultaneous (encoded) sources, source k = sum_s src_w[k][s] e_s / (hx hz) (host float32
 * [nsim][nsrc], e.g. Rademacher +-1 weights, Sec. 3.2).  Data arrays are complex64
 * [nfreq][nsources][nrcv] over the context's frequencies (host or device). */
typedef struct {
    const int* src_idx;
    int nsrc;
    const float* src_w;     /* [nsim][nsrc] or NULL */
    int nsim;
    const int* rcv_idx;
    int nrcv;
} fwi_survey;

/* d = P^T H(m, w_j)^{-1} q_k for every frequency and source of the survey (the synthetic
 * data of Eq. 3.3); *iters_out (may be NULL) receives the Helmholtz iterations used. */
int fwi_forward_data(helm_ctx* ctx, const fwi_survey* survey, double tol, helm_c64* d_out, long long* iters_out);

/* Sensitivity products (Eq. 3.10 written out from the operator of Eq. 3.1: dH/dm =
 * -w^2 (1 - i gamma)), for real model perturbations of m = kappa^2:
 *   fwi_jacobian:          dd = J dm,  dd_jk = P^T w_j^2 H^{-1} ((1 - i gamma) u_jk dm)
 *   fwi_jacobian_adjoint:  dm = J^T dd = Re(J^H dd) = sum_jk w_j^2 Re((1 - i gamma) u_jk mu_jk),
 *                          H mu_jk = P conj(dd_jk)   (conjugation identity, Sec. 4.3)
 * dm : float32 [nz][nx]; dd : complex64 [nfreq][nsources][nrcv]; host or device.  Each call
 * solves for the forward fields (tolerance tol) and then the sensitivity or adjoint
 * systems (same tolerance; the paper takes 1e-4 for these). */
int fwi_jacobian(helm_ctx* ctx, const fwi_survey* survey, const float* dm, double tol, helm_c64* dd_out);
int fwi_jacobian_adjoint(helm_ctx* ctx, const fwi_survey* survey, const helm_c64* dd, double tol, float* dm_out);

typedef struct {
    double tol;             /* forward and adjoint solves (misfit, gradient)          (1e-6) */
    double tol_sens;        /* sensitivity solves inside conjugate gradients           (1e-4) */
    int    cg_iters;        /* conjugate-gradient steps on the Gauss-Newton system       (5) */
    float  reg;             /* Tikhonov term reg I added to J^T J                        (0) */
    float  m_min, m_max;    /* bounds of m = kappa^2 after the step              (0, 1e30) */
    int    max_backtracks;  /* halvings of the step when the objective does not drop   (4) */
    int    reg_kind;        /* regulariser R of Sec. 5.1 on v = m - m_ref: 0 none, 1 R_diff =
                               ||grad_h v||^2, 2 R_high = ||Lap_h v||^2, Lap_h = -grad_h^T grad_h
                               (forward differences on the interior edges, scaled by 1/hx, 1/hz)  (0) */
    float  alpha;           /* weight of R: the objective is Phi(m) + alpha R(m)            (0) */
    const float* m_ref;     /* reference model [nz][nx], host or device; NULL: zero     (NULL) */
} fwi_gn_opts;
typedef struct {
    double misfit_before, misfit_after;   /* Eq. 3.5 at the model before / after the step */
    double step;                          /* accepted step length (0: model unchanged)    */
    int    cg_iters;                      /* CG steps taken                               */
    long long iters_forward, iters_adjoint, iters_sensitivity, iters_line_search;
                                          /* Helmholtz (FGMRES) iterations per phase      */
    double objective_before, objective_after;   /* Phi + alpha R before / after the step */
} fwi_gn_info;
void fwi_default_gn_opts(fwi_gn_opts* opts);
/* kappa = sqrt(m) for n nodes (device arrays): the medium of a model m = kappa^2. */
int fwi_model_to_kappa(const float* m, float* kappa, long long n);
/* One Gauss-Newton iteration of Alg. 1 at the context's frequencies for the objective
 * Phi(m) + alpha R(m) (Eq. 3.5 and a regulariser of Sec. 5.1): sets the medium from m
 * (clipped to [m_min, m_max]; kappa = sqrt(m), gamma kept), forward fields and the misfit
 * Phi, the gradient 2 J^T r + alpha grad R, cg_iters conjugate-gradient steps on
 * (J^T J + alpha K + reg I) dm = -(J^T r + alpha K (m - m_ref)) from 0 (K = -Lap_h for
 * R_diff, Lap_h^2 for R_high) with the forward fields kept (two solves per source and
 * frequency per step), then m <- clip(m + a dm) for a = 1, 1/2, ... (at most
 * max_backtracks halvings) as soon as the objective drops; if none does, m is unchanged.
 * info->misfit_* report Phi, info->objective_* Phi + alpha R.
 * d_obs: complex64 [nfreq][nsrc][nrcv] per POINT source (host or device); with
 * simultaneous sources it is encoded here with the survey's weights (d_k = sum_s w_ks d_s).
 * m: float32 [nz][nx] (host or device), updated in place; the context's medium is left
 * at the returned m.  Memory: 16 bytes per grid point per (frequency, source) for the
 * kept fields. */
int fwi_gn_iteration(helm_ctx* ctx, const fwi_survey* survey, const helm_c64* d_obs, const fwi_gn_opts* opts,
                     float* m, fwi_gn_info* info);

/* ---- several grids (per-frequency grids of the FWI windows) ------------------------------
 * helm_resample: dst = alpha * bilinear(src) + beta * dst between two node grids covering the
 * same rectangle (node (i, j) of an n_x x n_z grid at the cell centre ((i + 1/2) Lx / n_x,
 * (j + 1/2) Lz / n_z); source positions clamped to its outermost nodes).  float32 device
 * arrays [nz0][nx0] -> [nz1][nx1], not aliased; issued on `stream` (cudaStream_t) and waited
 * for.  With beta = 1 it adds a resampled update to a field. */
int helm_resample(const float* src, int nx0, int nz0, float* dst, int nx1, int nz1, float alpha, float beta,
                  void* stream);
/* helm_solve for several contexts in one call (different grids, media or frequencies):
 * context i solves its nrhs[i] right-hand sides rhs[i] into x[i] (freq_idx[i] may be NULL,
 * freq_idx itself may be NULL; stats may be NULL or an array of nctx), each from its own host
 * thread on its context's stream, so that contexts with distinct streams share the GPU.
 * A context may appear once.  Returns the first hard error, else HELM_ENOCONV /
 * HELM_EBREAKDOWN if some context had them, else HELM_OK; helm_last_error() names the
 * context. */
int helm_solve_multi(helm_ctx* const* ctxs, int nctx, const helm_c64* const* rhs, helm_c128* const* x,
                     const int* nrhs, const int* const* freq_idx, double tol, int flags, helm_stats* stats);

void helm_destroy(helm_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Encoder-solver network (Sec. 3.4, Eq. 3.13-3.14, 4.1; Fig. 1 caption).
 * Two U-Nets of `levels` levels with widths[0..levels-1] channels (multiples of
 * 16, at most 128).  A ResNet layer is relu(x + conv(relu(conv(x)))).  Encoder
 * (input [c_ref kappa, gamma, w h kappa], c_ref = 1500 m/s): in conv, 2 ResNet
 * layers per level with a stride-2 conv between levels; on the way up a
 * nearest-x2 + conv, concatenation with the level's feature, a conv back to
 * the level's width and one ResNet layer, giving the context z_l of each level.
 * Solver (input [Re r^, Im r^, gamma], r^ = r / rms(r)): the same shape, with
 * the context z_l concatenated (and reduced by a conv) at every level of the
 * way down, and an output conv to 2 channels.  The preconditioner (Eq. 3.14)
 * is M_VU(r) = V-cycle(e_0, r) with e_0 = h^2 rms(r) (out_0 + i out_1), composed as
 * e_0 + V(r - H e_0) (exact when e_0 = H^-1 r), and for a RHS whose restart cycles stall
 * a e_0 + V(r - a H e_0) with a = <H e_0, r> / <H e_0, H e_0> when the network's step would
 * raise the residual (opts.cnn_vcycle = 2, default; 0, 1 and 3 select one composition).
 * Outside a solve, composition 2 is the plain one.
 * Convolutions are 3x3 implicit GEMMs on the tensor cores (tcgen05, BF16
 * operands, FP32 accumulation in tensor memory).
 * Parameters are one flat FP32 vector: per layer weights [cout][9][cin] then
 * bias [cout], layers in the order above (encoder, then solver).
 * ------------------------------------------------------------------------- */
/* Create the network with seeded He-normal initial weights (cnn_init_params with gain
 * 0.5: the half-scale initialisation the training starts from) and zero biases. */
int cnn_create(cnn_model** out, int levels, const int* widths, unsigned long long seed);
void cnn_destroy(cnn_model* net);
long long cnn_num_params(const cnn_model* net);
/* Load / read the FP32 parameters (host or device pointer, n = cnn_num_params). */
int cnn_set_params(cnn_model* net, const float* params, long long n);
/* Seeded He-normal initial weights, std = gain * sqrt(2 / (9 C_in)) per layer,
 * zero biases (normal draws by Box-Muller from splitmix64 started at seed). */
int cnn_init_params(cnn_model* net, unsigned long long seed, float gain);
int cnn_get_params(const cnn_model* net, float* params, long long n);
/* Raw network forward (inputs rounded to BF16): enc_in FP32 [nenc][ny][nx][3],
 * sol_in FP32 [nsol][ny][nx][3], out FP32 [nsol][ny][nx][2].  nenc is 1 (every
 * solver image uses the one context) or nsol (image i uses context i).
 * ny, nx divisible by 2^(levels-1).  Host or device pointers. */
int cnn_forward(cnn_model* net, const float* enc_in, int nenc, const float* sol_in, int nsol, int ny, int nx,
                float* out);
/* The network preconditioner of a context created with a network (Eq. 3.14):
 * e = M_VU(r) (composed as opts.cnn_vcycle selects) for with_vcycle = 1, or
 * e = e_0 = h^2 rms(r) net(r / rms(r)) for with_vcycle = 0.
 * r, e : complex64 [nrhs][nz][nx] (host or device); freq_idx as in helm_solve. */
int cnn_precond_apply(helm_ctx* ctx, const helm_c64* r, helm_c64* e, int nrhs, const int* freq_idx,
                      int with_vcycle);
/* ---- training (Sec. 4.1-4.2, Eq. 4.2-4.3, Alg. 2) ---------------------------------
 * Data of Eq. 4.3 for the context's medium: b = H x, x~ = FGMRES(H, M = V-cycle, b, 0)
 * after exactly iters[i] steps (1 <= iters[i] <= restart), r = b - H x~, e = x - x~.
 *   x : complex64 [nb][nz][nx], the caller's draws of x ~ CN(0, 1); iters : host int32 [nb]
 *   r_out, e_out : complex64 [nb][nz][nx]; nb <= max_rhs.  Host or device pointers. */
int cnn_make_samples(helm_ctx* ctx, const helm_c64* x, const int* freq_idx, const int* iters, int nb,
                     helm_c64* r_out, helm_c64* e_out);
/* One data step of Alg. 2 for every pair (r, e): e_net = network(r) (the error estimate,
 * without V-cycle), e~ = FGMRES(H, V-cycle, r, x0 = e_net) after one step, and the new pair
 * (r - H e~, e - e~) (literal = 0, the residual-correction reading) or (H e~, e~) (literal = 1,
 * Alg. 2 as printed).  Needs a context created with a network. */
int cnn_refine_samples(helm_ctx* ctx, const helm_c64* r, const helm_c64* e, const int* freq_idx, int nb,
                       int literal, helm_c64* r_out, helm_c64* e_out);
/* MSE loss of Eq. 4.2 on a batch, (1/nb) sum ||e_net(r_i) - e_i||^2 with
 * e_net = h^2 rms(r) net(r / rms(r)) (network output only, no V-cycle), and its gradient
 * with respect to every parameter (flat, FP32, written to grad_out if not NULL; host or
 * device).  The context supplies the medium and frequencies (freq_idx per pair). */
int cnn_loss_grad(cnn_model* net, helm_ctx* ctx, const helm_c64* r, const helm_c64* e, const int* freq_idx,
                  int nb, double* loss, float* grad_out);
/* One Adam step (Kingma & Ba; beta = (0.9, 0.999), eps = 1e-8, learning rate lr) on the loss
 * of cnn_loss_grad; returns the loss before the step.  If the context was created with
 * this network its context features are recomputed with the new weights. */
int cnn_train_step(cnn_model* net, helm_ctx* ctx, const helm_c64* r, const helm_c64* e, const int* freq_idx,
                   int nb, float lr, double* loss);
int cnn_adam_reset(cnn_model* net);
/* Training loss of cnn_loss_grad / cnn_train_step: kind 0 (default) is Eq. 4.2,
 * (1/m) sum_i ||e_net,i - e_i||^2; kind 1 weighs each sample by 1 / ||e_i||^2
 * (relative error), so that the small, smooth errors left after several
 * preconditioned GMRES steps count as much as the large ones.  HELM_EINVAL for
 * other kinds. */
int cnn_set_loss(cnn_model* net, int kind);

/* ---- retraining inside the library: Alg. 2 of Sec. 4.2, one unit per call ----------
 * The context (created with the network) owns a dataset of (residual, error) pairs of
 * its medium and a schedule:
 *   - the first cnn_retrain_step builds initial_size pairs by Eq. 4.3 (x ~ CN(0, 1),
 *     b = H x, x~ after k V-cycle-preconditioned FGMRES steps, k uniform on
 *     [1, max_gmres_steps], pair (b - H x~, x - x~)); pair i has frequency index i mod nfreq;
 *   - every call trains on the next `batch` pairs of the current epoch (a fresh
 *     permutation per epoch; the last batch of an epoch may be shorter): one Adam step
 *     of cnn_train_step with learning rate lr (the caller schedules lr);
 *   - at the end of each of the first data_epochs epochs every pair gets a refined
 *     partner (cnn_refine_samples: the network's estimate followed by one preconditioned
 *     GMRES step), doubling the dataset: 128 -> 1024 pairs over 3 epochs by default.
 * Steps continue past `epochs` on the full dataset; cnn_retrain_state reports done = 1 then.
 * Random draws (x, k, the permutations) come from a counter-based splitmix64 stream of
 * `seed` (Steele, Lea and Flood 2014), so a run is reproducible.  The dataset takes
 * 2 x 8 bytes per grid point per pair (8.6 GB for 1024 pairs of 1024 x 512). */
typedef struct {
    int initial_size;            /* pairs of the initial dataset, Eq. 4.3            (128) */
    int data_epochs;             /* epochs that end with the data step of Alg. 2       (3) */
    int epochs;                  /* epochs of the schedule                             (30) */
    int max_gmres_steps;         /* largest step count of Eq. 4.3 (<= restart)          (10) */
    int literal;                 /* 1: Alg. 2's pair as printed (H e~, e~); 0: residual-correction
                                    pair (r - H e~, e - e~)                              (0) */
    unsigned long long seed;     /* generator seed                                        (3) */
} cnn_retrain_opts;
void cnn_retrain_default_opts(cnn_retrain_opts* opts);
/* (Re)start the schedule with the given options (NULL: defaults), dropping any dataset.
 * HELM_EINVAL without a network or for out-of-range options; HELM_ENOMEM if the dataset
 * does not fit.  cnn_retrain_step starts with the defaults when this was not called. */
int cnn_retrain_begin(helm_ctx* ctx, const cnn_retrain_opts* opts);
/* One unit of Alg. 2 (see above); loss_out (host, may be NULL) receives the batch loss of
 * Eq. 4.2 (or its relative form, cnn_set_loss) before the Adam step.  The context must
 * have been created with `net`; 1 <= batch <= max_rhs. */
int cnn_retrain_step(cnn_model* net, helm_ctx* ctx, int batch, float lr, float* loss_out);
/* out6 = {epochs completed, pairs of the current epoch trained on, dataset size,
 * Adam steps taken, done (epochs reached), dataset capacity}; zeros before the first step. */
int cnn_retrain_state(const helm_ctx* ctx, long long* out6);
/* Copy pairs first .. first + n - 1 of the dataset (complex64 [n][nz][nx], host or
 * device) and their frequency indices (host int32 [n], may be NULL). */
int cnn_retrain_pairs(helm_ctx* ctx, int first, int n, helm_c64* r_out, helm_c64* e_out, int* freq_out);

/* ---- checkpoints of the network (trained weights outlive the process) ----------------
 * File: "HELMCNN1", then little-endian u32 version (1), u32 levels, u32 widths[8] (unused
 * slots 0), i64 number of parameters, i64 Adam steps, u32 flags (bit 0: Adam moments
 * follow), u32 loss kind, u64 FNV-1a checksum of the float payload, then the FP32
 * parameters (cnn_set_params layout) and, with bit 0, the Adam moments m and v.
 * cnn_load creates the network the file describes (the architecture comes from the
 * header) and returns HELM_EINVAL for a missing, truncated, corrupted (checksum) or
 * foreign file; cnn_save returns HELM_EINVAL if the file cannot be written. */
int cnn_save(const cnn_model* net, const char* path);
int cnn_load(cnn_model** out, const char* path);

/* One 3x3 convolution layer of the network, FP32 in and out (rounded to BF16 inside,
 * FP32 accumulation on the tensor cores, output rounded to BF16 then widened):
 *   y = act(bias + res + conv(concat(x0, x1)))      NHWC, weights [cout][9][c0 + c1]
 *   x0 [nb][hin][win][c0], x1 [nb or 1 (x1_bcast)][hin][win][c1] or NULL (c1 = 0),
 *   res [nb][hout][wout][cout] or NULL, mode 0 same / 1 stride-2 down / 2 nearest-x2 up,
 *   relu 0/1, cout <= 128; y [nb][hout][wout][cout].  Host or device pointers. */
int cnn_conv3x3(const float* x0, int c0, const float* x1, int c1, int x1_bcast, int nb, int hin, int win,
                const float* w, const float* bias, int cout, const float* res, int mode, int relu, float* y);

/* Backward pass of one 3x3 convolution layer (for parity tests and offline use):
 * for y = conv(concat(x0, x1)) (the layout of cnn_conv3x3, mode 0 same / 1 stride-2 down /
 * 2 nearest-x2 up) and an upstream gradient gy FP32 [nb][hout][wout][cout] (any ReLU mask
 * already applied), the input gradients gx0 [nb][hin][win][c0] and gx1 ([nb or 1 when
 * x1_bcast][hin][win][c1], summed over the images for a broadcast x1), the weight gradient
 * dw [cout][9][c0 + c1] and the bias gradient db [cout].  Inputs, weights and gy are rounded
 * to BF16; the products accumulate in FP32 on the tensor cores (the weight gradient on the
 * path of cnn_set_wgrad_path).  Outputs (host or device, any may be NULL) are overwritten.
 * c1 > 0 needs c0 % 16 == 0.  HELM_EINVAL for bad sizes. */
int cnn_conv3x3_backward(const float* x0, int c0, const float* x1, int c1, int x1_bcast, int nb, int hin, int win,
                         const float* w, int cout, int mode, const float* gy, float* gx0, float* gx1, float* dw,
                         float* db);
/* Which kernel computes the weight gradients of the backward pass: 0 (default) the
 * tensor cores (K = output pixels; per-CTA partial sums added in a fixed order, so the
 * result does not change from run to run), 1 the FP32 CUDA-core kernel (one atomic add
 * per weight per CTA; also the fallback for a layer the tensor-core kernel does not
 * take).  Process-wide.  HELM_EINVAL for any other value. */
int cnn_set_wgrad_path(int path);
/* Tile plan of the tensor-core weight gradient for a layer shape, computed on the host
 * (no GPU needed), for checking its bounds: mode 0/1/2 as above, c0, c1 input channels
 * (multiples of 8), npad output channels (a multiple of 16, at most 128), hin x win input
 * grid, nb images, sms multiprocessors (0: 148).  out20 = {K tiles, tile width, tile rows,
 * pixels per K tile, tiles along x, along y, output parities, input chunks per tap,
 * chunks from x0, chunks of the gradient, taps per group, groups, largest chunk count of
 * a group, bytes per staged plane, bytes per stage, stages, slack bytes after the ring,
 * TMEM columns, CTAs along K, dynamic shared memory bytes}.  HELM_EINVAL when the kernel
 * does not take the layer. */
int cnn_wgrad_plan(int mode, int c0, int c1, int npad, int hin, int win, int nb, int sms, long long* out20);

/* Which kernel runs the convolutions.  path 0 (default): the TMA halo-tile
 * kernel (the input tile of a CTA staged once, the nine taps read as shifted
 * shared-memory views), falling back to the gather kernel for a layer it
 * cannot take; path 1: the gather kernel for every layer; path 2: as path 0,
 * but same-grid layers with 16 output channels put the three column taps into
 * the MMA's N and add them in the epilogue (fewer shared-memory operand reads,
 * more epilogue work; slower than path 0 on GB300 so far); path 3: as path 0,
 * but same-grid layers with 16 or 32 output channels put the three tap rows into
 * the MMA's N (three MMAs of N = 48 or 96 per staged row and 16-channel group
 * instead of nine of N = 16 or 32 per output row) and add the three rows' partial
 * sums in the epilogue (Sec. 3.4's 3x3 convolutions; the tap sums are unchanged;
 * also slower than path 0 on GB300 so far).  Process-wide; for tests and
 * measurements.  Returns HELM_EINVAL for any other value. */
int cnn_set_conv_path(int path);
/* Autotuning of the convolutions' tiling.  Runs the network's solver pass once
 * on a synthetic residual batch of nrhs RHS (1 <= nrhs <= max_rhs) of the
 * context's medium.  The first launch of every layer shape times its candidate
 * tilings and records the fastest: the default stage and ring budgets,
 * 36/110, 56/112, 100/200 and 47/200 KB, at most 4 rows per tile, one
 * accumulator buffer of up to 512 TMEM columns (more M blocks per tile), for
 * 16-channel same-grid layers the column-taps-in-N variant, and for up layers a tile
 * per output row parity (default budgets, 100/200 KB, one buffer, one buffer with a
 * 200 KB ring).  Later launches of
 * that shape, at any batch size and in any context, use it.  The table is
 * process-wide; explicit cnn_set_conv_tiling / cnn_set_conv_ring values take
 * precedence.  Layers that accumulate into their output (the backward pass)
 * keep the defaults.  *n_shapes (may be NULL) receives the number of tuned
 * shapes.  HELM_EINVAL without a network or for nrhs outside the range. */
int cnn_autotune(helm_ctx* ctx, int nrhs, int* n_shapes);
/* Forget every tuned tiling. */
void cnn_autotune_reset(void);
/* Tile plan of the TMA convolution for a layer shape, computed on the host (no
 * GPU needed), for checking its bounds: mode 0 same grid, 1 stride-2 down, 2
 * nearest x2 up, 3 transpose of stride 2; c0, c1 input channels (multiples of
 * 16), npad output channels (16 or a multiple of 32, at most 128), hin x win
 * input grid, nb images; stage_kb / ring_kb / rows_cap as for
 * cnn_set_conv_ring / cnn_set_conv_tiling (0 = default); narrow = 1 selects the
 * column-taps-in-N variant for 16-channel same-grid layers, narrow = 2 the
 * row-taps-in-N variant for 16- and 32-channel ones, narrow = 3 the tiling with one
 * accumulator buffer of up to 512 TMEM columns (any mode; an autotuner candidate),
 * narrow = 4 an up layer with a tile per output row parity (cnn_set_conv_upsplit; 2
 * parities per tile, tiles counted per parity), narrow = 5 both of the last two.
 * out19 = {tiles,
 * tile width, tile rows, staged row pitch, M blocks per parity, parities,
 * parity sub-planes, plane bytes, parity stride bytes, weight bytes, stage
 * bytes, stages, TMEM columns, TMEM slots, slot columns, mode used (4 or 6 =
 * the variant), epilogue warpgroups and staged rows per commit of mode 6,
 * accumulator buffers}.  HELM_EINVAL for an invalid shape or one the kernel does not
 * take (out19 is filled either way for a valid shape). */
int cnn_conv_plan(int mode, int c0, int c1, int npad, int hin, int win, int nb, int stage_kb, int ring_kb,
                  int rows_cap, int narrow, int* out19);
/* Launches of the column-taps-in-N convolution since the library was loaded. */
long long cnn_conv_narrow_launches(void);
/* Launches of the row-taps-in-N convolution (cnn_set_conv_path(3)) since the library
 * was loaded. */
long long cnn_conv_rowtaps_launches(void);
/* Tile height limit of the TMA halo-tile kernel: at most max_rows output rows per
 * tile (0 = automatic: as many as two 128-column TMEM accumulator buffers and a
 * 47 KB stage allow).  Process-wide; for tuning.  HELM_EINVAL outside [0, 254]. */
int cnn_set_conv_tiling(int max_rows);
/* Accumulator buffers of the TMA halo-tile kernel (modes same, down, up and the
 * transpose of down): 1 = one TMEM buffer of up to 512 columns, twice the M blocks per
 * tile, the MMAs of a tile waiting for the previous tile's epilogue; 2 or 0 = the
 * default (two buffers, or the autotuned choice).  Process-wide; takes precedence over
 * the tuned table like the other tiling knobs.  HELM_EINVAL outside [0, 2]. */
int cnn_set_conv_buffers(int nbuf);
/* Tiling of the up layers (nearest x2 then a 3x3 convolution) in the TMA halo-tile
 * kernel: 1 = a tile computes one output row parity (its two column parities), so a
 * stage holds the 8 merged taps of that parity and a tile twice the rows; the tiles of
 * the two parities alternate.  0 = the default (all four parities per tile, or the
 * autotuned choice).  Process-wide; takes precedence over the tuned table like the other
 * tiling knobs.  HELM_EINVAL outside [0, 1]. */
int cnn_set_conv_upsplit(int on);
/* Shared-memory budgets of the TMA halo-tile kernel: at most stage_kb KB per
 * stage (one tile's 16-channel group plus its weights; taller tiles are cut
 * until a stage fits) and ring_kb KB for the ring of stages (2 to 6 stages; a
 * ring above about 110 KB leaves one CTA per SM).  0 keeps the default (47 and
 * 96 KB; 100 and 200 KB for stride-2 layers).  Process-wide; for tuning.  HELM_EINVAL for stage_kb outside
 * [0, 128], ring_kb outside [0, 200], or a ring smaller than a stage. */
int cnn_set_conv_ring(int stage_kb, int ring_kb);
/* Launch shape of the last TMA convolution, for diagnostics: out6 = {grid,
 * CTAs per SM, CTAs per SM that registers and shared memory allow,
 * dynamic shared memory per CTA in bytes, registers per thread, static shared
 * memory in bytes}. */
void cnn_conv_last_launch(int* out6);
/* Launches of each convolution kernel since the library was loaded (either
 * pointer may be NULL). */
void cnn_conv_launch_counts(long long* tma, long long* gather);

/* Per-kernel-class timing: when enabled, every kernel launch of the context is
 * bracketed by CUDA events on its stream and the main kernels add the
 * algorithmic bytes they move (the minimum DRAM traffic of their definition:
 * complex64 vectors read and written once per grid point, coefficients shared
 * by the batch not counted) to a device counter of their class.  Enabling
 * resets the totals.  helm_profile_read fills up to max entries of class names
 * (static strings), total milliseconds, launch counts and algorithmic bytes,
 * and the number of entries written (any output pointer may be NULL). */
int helm_profile_enable(helm_ctx* ctx, int on);
int helm_profile_read(helm_ctx* ctx, int max, const char** names, double* ms, long long* launches,
                      double* bytes, int* count);
/* Algorithmic flops per class since profiling was enabled, in the order of
 * helm_profile_read (nonzero for the tensor-core convolutions: 2 x 9 x C_in x
 * C_out per output pixel of every layer of the network's forward pass). */
int helm_profile_flops(helm_ctx* ctx, int max, double* flops, int* count);

/* CUDA graphs for the restart cycles of helm_solve (on by default).  With the
 * MG preconditioner or none, the second restart cycle of a solve is captured as
 * a CUDA graph (the k Arnoldi steps with their V-cycles, the update of x, the
 * true residual and the restart check) and every later cycle replays it with one
 * launch.  CNN-preconditioned solves and solves under the profiler run their
 * cycles as single launches; so does a solve whose capture fails.  Results are
 * the same either way.  HELM_EINVAL for a null context. */
int helm_set_graphs(helm_ctx* ctx, int on);

/* Autotuning of the multigrid sweeps' thread-block shapes (and, for a context with a
 * network, of the convolutions' tiling, cnn_autotune): runs one V-cycle on a synthetic batch
 * of nrhs right-hand sides (1 <= nrhs <= max_rhs).  The first Jacobi sweep on each grid times
 * the candidate block shapes (32x8, 64x4, 32x4, 128x2, 32x16, 16x16) with CUDA events and
 * records the fastest in a process-wide table that every later sweep on that grid uses, at
 * any batch size and in any context.  *n_shapes (may be NULL) receives the number of tuned
 * (sweep, grid) entries.  helm_setup runs it with max_rhs when opts.autotune is set. */
int helm_autotune(helm_ctx* ctx, int nrhs, int* n_shapes);
/* Forget every tuned block shape of the sweeps. */
void helm_autotune_reset(void);

/* Number of kernels the library has launched in this process (all contexts;
 * a graph replay counts the kernels it runs). */
long long helm_launch_count(void);

/* Thread-local description of the last error on this thread ("" if none). */
const char* helm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
