/*
 * fsi.h -- C ABI of the GB300 frequency-response library for coupled
 * shell-cavity (fluid-structure) finite-element models.
 *
 * The library computes the frequency sweep of the full-order model
 *     A(w) x(w) = f,   A(w) = K + i w D - w^2 M,   y(w) = C^T x(w)
 * (paper Sec. 2, Eq. 1-3, and Sec. 3.3, Eq. 8) on one GPU, and builds and
 * evaluates rational Arnoldi reduced models of it (Sec. 3.3, Eq. 9-11).
 *
 * Conventions for every entry point
 *   - Every function returns fsi_status: 0 on success, a negative code on
 *     error.  No exception or abort crosses the ABI.  fsi_last_error() gives a
 *     thread-local message for the last failure.
 *   - Frequencies are in Hz, FP64, host memory.  w = 2 pi f.
 *   - "device" pointers are CUDA global-memory pointers of the current device;
 *     "host" pointers are ordinary CPU memory.  The caller allocates and owns
 *     every buffer; the library allocates no device memory in these calls (the
 *     workspace is the caller's).  Streams are borrowed (cudaStream_t as void*,
 *     NULL = legacy default stream).  Calls are asynchronous on that stream
 *     unless stated; any call that returns host-visible results synchronizes it.
 *   - Complex numbers are fsi_c64 {re, im} pairs of doubles (complex128
 *     layout).  Matrices are column-major unless stated: F[col * n + i].
 *   - DoF numbering is slab major: slab k (nodes with z-index k) holds first the
 *     nx*ny pressure DoFs, index i + nx*j, then (w, beta_s, beta_z) of every
 *     shell ring node (ring numbered counter-clockwise from grid node (0, 0)).
 *     Global index = k * b + local, b = nx*ny + 3*n_ring.
 *   - On an error a sweep has completed and written every frequency batch
 *     before the failing one (stats->n_done frequencies); nothing after it.
 */
#ifndef FSI_H
#define FSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } fsi_c64;

typedef enum {
    FSI_OK = 0,
    FSI_EINVAL = -1,      /* bad argument (sizes, pointers, options)                */
    FSI_ENOMEM = -2,      /* workspace or model buffer smaller than required        */
    FSI_ECUDA = -3,       /* a CUDA runtime call failed (message has the CUDA text) */
    FSI_ESINGULAR = -4,   /* zero or non-finite pivot in a factorisation            */
    FSI_ENOCONV = -5,     /* refinement did not reach the tolerance in max_refine   */
    FSI_ETIMEOUT = -6,    /* a bounded device wait gave up                          */
    FSI_ESTATE = -7       /* call out of order (e.g. reduced model not built)       */
} fsi_status;

typedef enum {
    FSI_FP64 = 0,         /* factor and solve in FP64 (the plain full-order sweep)  */
    FSI_FP32_IR = 1,      /* factor in FP32, FP64 residual iterative refinement     */
    FSI_BF16X6_IR = 2,    /* as FSI_FP32_IR, the long trailing updates on the tensor */
                          /* cores: tcgen05 BF16 MMAs on three-plane splits of the   */
                          /* FP32 operands (six products, FP32-level accuracy),      */
                          /* accumulations of 64 elements drained into FP32 sums     */
    FSI_BF16_IR = 3       /* as FSI_BF16X6_IR with one BF16 plane (one product):    */
                          /* a BF16 factor with FP32 accumulation, refined in FP64   */
} fsi_precision;

/* Geometry and materials of the coupled model (paper Sec. 2; loss factor
 * Sec. 3.3 after Eq. 8).  All host memory; eta has n_eta = 1 (uniform) or
 * nz - 1 (one per shell element layer between slabs k and k+1) entries. */
typedef struct {
    double Lx, Ly, Lz;            /* cavity box, m                                  */
    int nx, ny, nz;               /* pressure nodes per direction (>= 3 each)       */
    double c, rho;                /* air: speed of sound m/s, density kg/m^3        */
    double E, nu, rho_s, t;       /* shell: Young's modulus, Poisson, density, m    */
    const double* eta;            /* shell loss factor(s), host                      */
    int n_eta;
    int has_floor;                /* 1: locally reacting impedance on face y = 0   */
    double Z_re, Z_im;            /* floor impedance, Pa s / m                       */
} fsi_model_desc;

/* Sizes derived from a description by fsi_model_dims. */
typedef struct {
    int64_t n;                    /* total DoFs = b * nz                           */
    int b;                        /* DoFs per slab                                  */
    int nz;                       /* slabs                                          */
    int n_press_slab;             /* nx * ny                                        */
    int n_ring;                   /* shell ring nodes per slab                      */
    int64_t nnz;                  /* nonzeros of the shared CSR pattern of K, M, D */
    size_t model_bytes;           /* size of the device model buffer                */
    double rho;                   /* copied from the description                    */
} fsi_dims;

/* Compute sizes.  Host only, no CUDA call.  Errors: FSI_EINVAL. */
fsi_status fsi_model_dims(const fsi_model_desc* desc, fsi_dims* out);

/* Assemble K (complex), M (real), D (complex) on the host into caller-owned
 * HOST arrays sharing one CSR pattern (paper Sec. 2, Eq. 1-3, coupling Eq. 5;
 * D from the floor impedance, Eq. 8): rowptr[n+1], col[nnz] (sorted within
 * each row), K[nnz], M[nnz], D[nnz].  No CUDA call.  Errors: FSI_EINVAL. */
fsi_status fsi_assemble_host(const fsi_model_desc* desc, int32_t* rowptr, int32_t* col,
                             fsi_c64* K, double* M, fsi_c64* D);

/* Assemble and upload into a caller-allocated DEVICE buffer of at least
 * dims.model_bytes bytes (256-byte aligned), on `stream`; synchronizes the
 * stream before returning.  The buffer's layout is private to the library.
 * Errors: FSI_EINVAL, FSI_ENOMEM (buffer too small), FSI_ECUDA. */
fsi_status fsi_assemble(const fsi_model_desc* desc, void* d_model, size_t model_bytes,
                        void* stream);

typedef struct {
    int precision;                /* fsi_precision                                   */
    int batch;                    /* frequencies factored together (>= 1)            */
    int max_refine;               /* refinement iterations cap (FP32_IR)             */
    double tol;                   /* target relative residual in the scaled norm    */
    int host_io;                  /* 1: F, rcv, p_out, spl_out are HOST pointers;   */
                                  /*    the copies happen inside the call           */
    int profile;                  /* 1: time every kernel launch with CUDA events   */
                                  /*    on `stream` and report per-kernel totals    */
    int refine;                   /* FSI_REFINE_IR or FSI_REFINE_GMRES              */
    int restart;                  /* GMRES restart length (0: 20)                   */
} fsi_solve_opts;

/* Refinement of the low-precision factor's solution against the FP64 residual:
 * plain refinement x <- x + LU^-1 r (converges when cond(A) u_low < 1), or
 * flexible GMRES on the FP64 system right-preconditioned by the factor (the
 * GMRES of paper Sec. 3.2 used as refinement), which also converges at the low
 * frequencies where the thin shell drives cond(A) to 1e7-1e8.  max_refine
 * caps the number of preconditioned solves in both cases. */
enum { FSI_REFINE_IR = 0, FSI_REFINE_GMRES = 1 };

/* Kernel classes of the per-kernel totals in fsi_sweep_stats. */
enum {
    FSI_K_GEMM = 0,               /* complex GEMM updates of the band LU (FP32/FP64 pipe) */
    FSI_K_PANEL = 1,              /* panel LU with partial pivoting                 */
    FSI_K_TRSM = 2,               /* unit-lower triangular solve of pivot rows      */
    FSI_K_LASWP = 3,              /* row interchanges                               */
    FSI_K_FORM = 4,               /* dense scaled rows of A(w) from the CSR values  */
    FSI_K_SHIFT = 5,              /* factor store write-out and window shift        */
    FSI_K_SOLVE = 6,              /* triangles of the forward / backward slab solves */
    FSI_K_RESID = 7,              /* FP64 residual, refinement updates, receivers   */
    FSI_K_GEMV = 8,               /* off-diagonal factor blocks in the slab solves  */
    FSI_K_PACK = 9,               /* hi/lo operand split of the tensor-core updates */
    FSI_K_TCGEMM = 10,            /* trailing updates on the tcgen05 tensor cores    */
    FSI_K_COUNT = 11,
    FSI_K_SLOTS = 12              /* array length in fsi_sweep_stats (room to grow) */
};

typedef struct {
    int n_done;                   /* frequencies completed                          */
    int max_iters;                /* largest refinement count over frequencies      */
    double max_relres;            /* largest final relative residual                */
    int n_unconverged;            /* frequencies above tol after max_refine         */
    int64_t launches;             /* kernel launches made by the call               */
    /* with opts.profile: summed event time (ms), algorithmic real flops (complex  */
    /* multiply-add = 8) and launch count per kernel class FSI_K_*                  */
    double kernel_ms[FSI_K_SLOTS];
    double kernel_flops[FSI_K_SLOTS];
    int64_t kernel_launches[FSI_K_SLOTS];
} fsi_sweep_stats;

/* Workspace bytes needed by frf_sweep_full for these options.  Host only. */
fsi_status frf_sweep_workspace(const fsi_dims* dims, const fsi_solve_opts* opts, int nrhs,
                               int nrcv, size_t* bytes);

/* Full-order frequency sweep (paper Sec. 2, Eq. 1; Sec. 3.3, Eq. 8): for every
 * frequency solve A(w) X = F by a block-banded LU with partial pivoting across
 * the stacked 2b x b panel of consecutive slabs, batched over `opts.batch`
 * frequencies, then refine in FP64 (FSI_FP32_IR) and read the receivers.
 *   d_model   device buffer filled by fsi_assemble
 *   f_hz      host, nf frequencies
 *   F         n x nrhs loads, column-major (device, or host if opts.host_io)
 *   rcv       nrcv receiver DoF indices (device or host)
 *   ws        device workspace of ws_bytes >= frf_sweep_workspace(...)
 *   p_out     [nf][nrcv][nrhs] complex pressures (device or host)
 *   spl_out   [nf][nrcv][nrhs] SPL, 20 log10(|p| / (sqrt(2) 20 uPa)), nullable
 *   iters_out host [nf] refinement iterations per frequency, nullable
 *   relres_out host [nf] final relative residual per frequency, nullable
 *   stats     host, nullable
 * Synchronizes the stream.  Errors: FSI_EINVAL, FSI_ENOMEM, FSI_ECUDA,
 * FSI_ESINGULAR, FSI_ENOCONV (results are still written). */
fsi_status frf_sweep_full(const fsi_dims* dims, const void* d_model, const double* f_hz, int nf,
                          const fsi_c64* F, int nrhs, const int32_t* rcv, int nrcv,
                          const fsi_solve_opts* opts, void* ws, size_t ws_bytes,
                          fsi_c64* p_out, double* spl_out, int32_t* iters_out,
                          double* relres_out, fsi_sweep_stats* stats, void* stream);

/* Residual R = F - A(w_f) X_f in FP64 for nf frequencies (the refinement's
 * residual kernel, paper Eq. 8 operator).  Device arrays: X and R are
 * [nf][nrhs][n] (for each frequency, column-major n x nrhs); F is n x nrhs.
 * f_hz host.  Errors: FSI_EINVAL, FSI_ECUDA. */
fsi_status fsi_residual(const fsi_dims* dims, const void* d_model, const double* f_hz, int nf,
                        const fsi_c64* X, const fsi_c64* F, int nrhs, fsi_c64* R, void* stream);

/* Batched partial LU with partial pivoting (the factorisation kernel set used
 * by every solve here), exposed for testing: for each of `batch` row-major
 * matrices A_i (m x ncols, leading dimension ld >= ncols, stride sA elements
 * between matrices) eliminate the first npiv columns, npiv <= min(m, ncols):
 * afterwards rows 0..npiv-1 hold L\U of the pivot block and U's remaining
 * columns, rows npiv..m-1 hold the multipliers (cols < npiv) and the Schur
 * complement (cols >= npiv); ipiv[i*npiv + j] is the row swapped with row j
 * (LAPACK getrf convention, 0-based).  precision selects FP64 or FP32 data:
 * A points to fsi_c64 (FP64) or to {float re, im} pairs (FSI_FP32_IR, and
 * FSI_BF16X6_IR / FSI_BF16_IR with the large trailing updates on the tensor
 * cores; those need ld, sA and the first column right of each update even,
 * otherwise they run on the FP32 SIMT pipe).  ws: device workspace of fsi_lu_workspace
 * bytes for the same precision and sizes.  n_singular_out (host, nullable)
 * gets the number of matrices that met a zero or non-finite pivot.  Any other
 * precision value is rejected with FSI_EINVAL.  The tensor-core precisions
 * synchronize the stream and returns FSI_ETIMEOUT when a bounded wait of a tensor-core
 * kernel gave up (see fsi_set_wait_limit); the factors are then invalid. */
fsi_status fsi_lu_workspace(int precision, int batch, int m, int ncols, int npiv, size_t* bytes);
fsi_status fsi_batched_lu(int precision, int batch, int m, int ncols, int npiv, void* A, int64_t ld,
                          int64_t sA, int32_t* ipiv, void* ws, size_t ws_bytes,
                          int* n_singular_out, void* stream);

/* Spin limit of the bounded mbarrier waits in the tensor-core kernels: the
 * number of polls after which a kernel gives up, records FSI_ETIMEOUT, waits
 * for the loads and MMAs it already issued and releases its tensor memory.
 * Each poll suspends the waiting thread for at most 4 us (it resumes as soon
 * as the awaited phase completes).  0 restores the default (about 4.2e6
 * polls, at most ~17 s); small values make the waits run out on purpose
 * (tests of the timeout path).  Process-wide, host only.  Errors: FSI_EINVAL
 * (negative). */
fsi_status fsi_set_wait_limit(int64_t spins);

/* Allocation-free variant of fsi_batched_lu (the paper has no counterpart; it
 * is a service to callers).  Some callers cannot allocate device memory: code
 * inside a memory pool that forbids new allocations, real-time loops that must
 * not wait on an allocator, or hosts whose interface has no way to pass a
 * workspace.  This entry point takes no workspace and calls no allocator
 * (no cudaMalloc, cudaFree or allocating library routine).  The kernels'
 * scratch (one pivot-status flag per matrix and a counter) lives in a fixed
 * 16 KiB device array inside the library, which every GPU that loads the
 * library holds until the process exits.
 *   - batch is limited to 4095 matrices; larger batches return FSI_EINVAL
 *     with a message (split the call, or use fsi_batched_lu).
 *   - precision is FSI_FP64 or FSI_FP32_IR.  FSI_BF16X6_IR and FSI_BF16_IR are rejected
 *     with FSI_EINVAL: their tensor-core updates need an operand workspace
 *     that grows with the matrices (use fsi_batched_lu).  Other values are
 *     rejected too.
 *   - Every call looks up the array's device address for the current device
 *     (a host-side lookup, no allocation).  The first call on a device also
 *     loads the library's device code there: make it before any stream
 *     capture.
 *   - All calls share the one array and each call clears the part it uses
 *     before use: calls that overlap on the GPU (different streams, or
 *     different host threads on one device) race and must be serialised.
 * Otherwise arguments, results and errors are those of fsi_batched_lu; it
 * synchronizes the stream when n_singular_out is not NULL. */
fsi_status fsi_batched_lu_noalloc(int precision, int batch, int m, int ncols, int npiv, void* A,
                                  int64_t ld, int64_t sA, int32_t* ipiv, int* n_singular_out,
                                  void* stream);

typedef struct {
    int precision;                /* factorisation per expansion point: FSI_FP64,  */
                                  /* FSI_FP32_IR or FSI_BF16X6_IR                   */
    int max_refine;               /* refinement cap per moment solve               */
    double tol;                   /* refinement tolerance per moment solve         */
    int second_order;             /* -1 auto (Eq. 9 if D != 0, else Eq. 10), 0, 1 */
    int batch_shifts;             /* expansion points factored, and their Eq. 10   */
                                  /* moments solved, together (0 or 1: one at a    */
                                  /* time; at most 64; Eq. 9 runs one at a time)   */
} fsi_rom_opts;

/* Workspace bytes for rom_build. */
fsi_status rom_workspace(const fsi_dims* dims, int nrhs, int q, int kmax, const fsi_rom_opts* opts,
                         size_t* bytes);

/* Rational Arnoldi basis (paper Sec. 3.3): for each expansion point w_j the
 * shifted matrix Kt_j = A(w_j) is factored once (Sec. 3.3, offline phase) and
 * q moments per load column are generated: Eq. 10 (first order,
 * Kt_j^-1 M) when the model has no damping matrix, Eq. 9 (second order, SOAR
 * recurrence with Dt_j = 2 i w_j M + D) otherwise.  Each new vector is
 * orthonormalised against all accepted ones by two classical Gram-Schmidt
 * passes (CGS2) and dropped if its norm falls below 1e-10 of its norm before
 * them.  F: device n x nrhs.  V: device n x kmax column-major (output, first
 * *k_out columns valid).  Errors: FSI_EINVAL, FSI_ENOMEM, FSI_ECUDA,
 * FSI_ESINGULAR. */
fsi_status rom_build(const fsi_dims* dims, const void* d_model, const double* shifts_hz, int nshift,
                     int q, const fsi_c64* F, int nrhs, int kmax, const fsi_rom_opts* opts,
                     void* ws, size_t ws_bytes, fsi_c64* V, int* k_out, void* stream);

/* Galerkin projection (text after Eq. 11): K_R = V^H K V, D_R = V^H D V,
 * M_R = V^H M V (k x k), f_R = V^H F (k x nrhs), C_R = rows rcv of V
 * (nrcv x k).  All device, column-major.  ws: device workspace of at least
 * n * k * 16 bytes. */
fsi_status rom_project(const fsi_dims* dims, const void* d_model, const fsi_c64* V, int k,
                       const fsi_c64* F, int nrhs, const int32_t* rcv, int nrcv, void* ws,
                       size_t ws_bytes, fsi_c64* KR, fsi_c64* DR, fsi_c64* MR, fsi_c64* fR,
                       fsi_c64* CR, void* stream);

/* Workspace bytes for rom_sweep with this precision (FSI_FP64 or FSI_FP32_IR). */
fsi_status rom_sweep_workspace(int k, int nrhs, int nrcv, int batch, int precision, size_t* bytes);

/* Reduced sweep (Eq. 11): y_R(w) = C_R (K_R + i w D_R - w^2 M_R)^-1 f_R for nf
 * frequencies, `batch` at a time.  Inputs device (column-major), f_hz host;
 * p_out [nf][nrcv][nrhs] device; spl_out same shape, nullable.
 *   precision FSI_FP64: each reduced system is equilibrated (row then column
 *     max scaling) and solved by dense LU with partial pivoting in FP64.
 *   precision FSI_FP32_IR (k <= 128, nrhs <= 4): the systems run through the
 *     persistent kernel of rom_multi_sweep (equilibrated LU in FP32, refined
 *     against the FP64 residual until the correction is at rounding level);
 *     a frequency whose refinement stalls is solved again by the FP64 path.
 *   fp64_out (host, nf, nullable): 1 where that FP64 re-solve happened.
 * The reduced model's error against the full-order model is not estimated
 * here: rom_greedy returns the residual estimate over its candidates and
 * rom_residual_check / rom_check_resolve evaluate the full-order residual.
 * Synchronizes the stream.  Errors: FSI_EINVAL, FSI_ENOMEM, FSI_ESINGULAR. */
fsi_status rom_sweep(int k, const fsi_c64* KR, const fsi_c64* DR, const fsi_c64* MR,
                     const fsi_c64* fR, const fsi_c64* CR, int nrhs, int nrcv,
                     const double* f_hz, int nf, int batch, int precision, void* ws,
                     size_t ws_bytes, fsi_c64* p_out, double* spl_out, int32_t* fp64_out,
                     void* stream);

/* Workspace bytes for rom_residual_check (batch frequencies at a time). */
fsi_status rom_residual_check_workspace(const fsi_dims* dims, int k, int nrhs, int batch, size_t* bytes);

/* Full-order FP64 residual of reduced solutions (the check of Sec. 3.3's error
 * measure by the residual, Sec. 5): for each frequency w = 2 pi f_hz[i] the reduced
 * system (K_R + i w D_R - w^2 M_R) x_R = f_R is solved as in rom_sweep, lifted to
 * x = V x_R and checked with the CSR residual of the full model:
 *   relres[i][c] = |f_c - A(w) x_c|_2 / |f_c|_2   (unscaled, FP64).
 * V: n x k column-major device basis the reduced matrices were projected with;
 * KR/DR/MR/fR as rom_project writes them (device, column-major); F: n x nrhs
 * column-major device loads; f_hz host; relres host [nf][nrhs].  nrhs <= 8.
 * Errors: FSI_EINVAL (sizes, small workspace), FSI_ESINGULAR (reduced system). */
fsi_status rom_residual_check(const fsi_dims* dims, const void* d_model, const fsi_c64* V, int k,
                              const fsi_c64* KR, const fsi_c64* DR, const fsi_c64* MR,
                              const fsi_c64* fR, const fsi_c64* F, int nrhs, const double* f_hz,
                              int nf, int batch, void* ws, size_t ws_bytes, double* relres,
                              void* stream);

/* Workspace bytes for rom_check_resolve (batch frequencies at a time; full:
 * the options of the full-order re-solves, host_io must be 0). */
fsi_status rom_check_resolve_workspace(const fsi_dims* dims, int k, int nrhs, int nrcv, int batch,
                                       const fsi_solve_opts* full, size_t* bytes);

/* Check and re-solve (paper Sec. 3.3: the reduced model's outputs are only as
 * good as its error check; the full-order solve stays the fallback).  p_out
 * and spl_out ([nf][nrcv][nrhs], device) hold the reduced outputs at f_hz
 * (e.g. from rom_sweep).  For every frequency the reduced solution is lifted,
 * x = V x_R, and judged by its full-order FP64 residual as rom_residual_check
 * computes it; a frequency whose largest relative residual over the load
 * columns exceeds res_tol is solved again at full order by frf_sweep_full with
 * the options `full` (device buffers), and its rows of p_out / spl_out are
 * replaced by the full-order outputs.  V, KR/DR/MR/fR, F, rcv: device, as for
 * rom_residual_check and frf_sweep_full.  Host outputs: relres_out [nf][nrhs]
 * (nullable), resolved_out [nf] (nullable; 1 where replaced), *n_resolved.
 * res_tol = 0 re-solves every frequency with a nonzero residual.
 * Synchronizes the stream.  Errors: FSI_EINVAL, FSI_ENOMEM, FSI_ECUDA,
 * FSI_ESINGULAR, FSI_ENOCONV (a re-solve missed its tolerance; outputs are
 * still written). */
fsi_status rom_check_resolve(const fsi_dims* dims, const void* d_model, const fsi_c64* V, int k,
                             const fsi_c64* KR, const fsi_c64* DR, const fsi_c64* MR,
                             const fsi_c64* fR, const fsi_c64* F, int nrhs, const int32_t* rcv,
                             int nrcv, const double* f_hz, int nf, int batch, double res_tol,
                             const fsi_solve_opts* full, void* ws, size_t ws_bytes, fsi_c64* p_out,
                             double* spl_out, double* relres_out, int32_t* resolved_out,
                             int* n_resolved, void* stream);

/* Reduced models on disk (the offline / online split of paper Sec. 3.3: the
 * reduced matrices are built once and reused).  A file holds nwin windows in
 * the slot layout of rom_windows (nwin = 1 and kmax = k for one model of
 * rom_project), their frequency ranges and expansion points, and optionally
 * the projection bases. */
typedef struct {
    int nwin;                     /* windows (1 for a single reduced model)        */
    int kmax;                     /* slot size of the matrix arrays                */
    int nrhs, nrcv;
    int64_t n;                    /* rows of the stored bases V; 0: none stored    */
    int nshift_total;             /* expansion points over all windows             */
} fsi_rom_info;

typedef struct {
    fsi_rom_info info;
    int on_device;                /* 1: the matrix arrays are device pointers,     */
                                  /* 0: host pointers                              */
    fsi_c64* KR;                  /* [nwin][kmax*kmax]: window w's k_w x k_w, ld k_w */
    fsi_c64* DR;
    fsi_c64* MR;
    fsi_c64* fR;                  /* [nwin][kmax*nrhs]: k_w x nrhs, ld k_w          */
    fsi_c64* CR;                  /* [nwin][kmax*nrcv]: nrcv x k_w, ld nrcv         */
    fsi_c64* V;                   /* [nwin][kmax*n]: n x k_w, ld n (NULL if n = 0)  */
    double* lo;                   /* host [nwin]: window frequency range, Hz        */
    double* hi;
    int32_t* k;                   /* host [nwin]: reduced order of each window      */
    int32_t* nshift;              /* host [nwin]: expansion points per window       */
    double* shifts_hz;            /* host [nshift_total], window after window       */
} fsi_rom_store;

/* Write the model described by `rom` to `path` (version-1 format, a 64-bit
 * checksum at the end); device arrays are staged through host memory on
 * `stream`.  Errors: FSI_EINVAL (sizes, NULL arrays, file not writable),
 * FSI_ECUDA. */
fsi_status rom_save(const char* path, const fsi_rom_store* rom, void* stream);

/* Sizes of the model in `path` (reads and checks the header only). */
fsi_status rom_file_info(const char* path, fsi_rom_info* info);

/* Read `path` into the caller's buffers: rom->info gives their capacity
 * (nwin, kmax, nshift_total at least the file's; nrhs, nrcv equal; n equal
 * when the file stores bases) and rom->on_device their kind.  Windows go to
 * the slots of rom->info.kmax; on success rom->info holds the file's sizes
 * with the caller's kmax, and lo / hi / k / nshift / shifts_hz are filled.
 * The data round-trips bit for bit.  Errors: FSI_EINVAL (not a model file,
 * unsupported version, truncated, checksum mismatch, buffers too small),
 * FSI_ECUDA. */
fsi_status rom_load(const char* path, fsi_rom_store* rom, void* stream);

/* Greedy expansion points (paper Sec. 3.3; its error measure replaced by a
 * residual estimate, as Sec. 5 suggests).  Options: */
typedef struct {
    int q;                        /* moments per load column per expansion point   */
    int kmax;                     /* basis columns at most (<= 1024)               */
    int max_shifts;               /* expansion points at most (initial included)  */
    double tol;                   /* stop when the largest estimate is <= tol      */
    fsi_rom_opts build;           /* factor precision / refinement of the moments */
    const float* mlp;             /* NULL, or device FSI_MLP_PARAMS of a trained
                                     estimator: the next point is the allowed
                                     candidate of largest predicted output error,
                                     kept only if its residual estimate is > tol
                                     (else the residual's argmax is taken)       */
} fsi_greedy_opts;

/* err[f] = |p[f] - p_ref[f]|_F / |p_ref[f]|_F over the nout outputs of each of
 * nf frequencies (the paper's relative output error; device arrays, p laid out
 * [nf][nout] as the sweeps write it). */
fsi_status rom_output_error(const fsi_c64* p_ref, const fsi_c64* p, int nf, int nout, double* err, void* stream);

/* Features of the learned estimator at each candidate (host arrays; X_out
 * ncand x 5 floats): (f - lo)/(hi - lo); the distances to the three nearest
 * expansion points over (hi - lo), capped at 1 and 1 where fewer exist;
 * log10(max(est, 1e-16)) / 4. */
fsi_status rom_features(const double* cand_hz, int ncand, const double* shifts_hz, int nshift,
                        const double* est, double lo, double hi, float* X_out);

/* Workspace bytes for rom_greedy (includes one rom_build workspace). */
fsi_status rom_greedy_workspace(const fsi_dims* dims, int nrhs, const fsi_greedy_opts* opts, size_t* bytes);

/* Builds the rational Arnoldi basis from init_hz (ninit points; 0: the middle
 * candidate), then repeatedly: projects (Galerkin, as rom_project), evaluates
 * at every candidate frequency the residual estimate
 *   est(w) = |R(w)(F - A(w) V x_R(w))|_F / |R(w) F|_F
 * (R(w): the full-order sweep's row equilibration; x_R: the reduced solution)
 * exactly from FP64 Gram blocks of [KV, DV, MV], and stops when max est <= tol,
 * at max_shifts points or at kmax columns; otherwise adds the candidate of
 * largest estimate (ties: lowest frequency) more than one candidate step away
 * from every existing point and appends its moments.  Candidates: host,
 * positive, strictly increasing.  F, V (n x kmax), KR/DR/MR (kmax x kmax
 * buffers; on return k x k, ld k), fR (k x nrhs, ld k), rcv, CR (nrcv x k):
 * device, column-major; rcv/CR may be NULL.  Host outputs: shifts_out
 * (max_shifts), *nshift_out, est_out (ncand; last estimates; nullable),
 * hist_out (max_shifts; largest estimate per round; nullable).  Errors:
 * FSI_EINVAL, FSI_ENOMEM, FSI_ECUDA, FSI_ESINGULAR. */
fsi_status rom_greedy(const fsi_dims* dims, const void* d_model, const fsi_c64* F, int nrhs,
                      const double* cand_hz, int ncand, const double* init_hz, int ninit,
                      const fsi_greedy_opts* opts, void* ws, size_t ws_bytes, fsi_c64* V, int* k_out,
                      fsi_c64* KR, fsi_c64* DR, fsi_c64* MR, fsi_c64* fR, const int32_t* rcv, int nrcv,
                      fsi_c64* CR, double* shifts_out, int* nshift_out, double* est_out, double* hist_out,
                      void* stream);

/* Local ROM windows (paper Sec. 3.3: one fROM per frequency window).  The
 * candidate band starts as one window with its own rom_greedy (initial points
 * at the window's quarter midpoints); a window whose greedy stops with its
 * largest estimate above greedy.tol is bisected (by candidate count), down to
 * min_points candidates, at most max_windows windows in all. */
typedef struct {
    fsi_greedy_opts greedy;       /* per window                                     */
    int max_windows;
    int min_points;               /* a window is not split below this many points  */
    int reuse;                    /* 1: a window split from a larger one starts from
                                     the larger windows' expansion points in its band,
                                     their Krylov blocks copied from a moment store
                                     (no new factorisation); 0: fresh points at the
                                     window's quarter midpoints                      */
    int init_points;              /* initial expansion points of a fresh window: the
                                     candidates nearest the midpoints of this many equal
                                     parts of it (0: 4, the quarter midpoints); with
                                     greedy.build.batch_shifts >= init_points they are
                                     factored and solved together                     */
    int init_windows;             /* the band starts as this many windows of equal
                                     candidate counts (0 or 1: one window)            */
} fsi_window_opts;

/* Workspace bytes for rom_windows (one greedy workspace + an n x kmax basis, and with
 * reuse a moment store of 4 * max_shifts * q * nrhs columns of n). */
fsi_status rom_windows_workspace(const fsi_dims* dims, int nrhs, const fsi_window_opts* opts, size_t* bytes);

/* Windows in increasing frequency order.  Device outputs, slot w of each:
 * KR/DR/MR at w*kmax*kmax (k_w x k_w, ld k_w), fR at w*kmax*nrhs (k_w x nrhs),
 * CR at w*nrcv*kmax (nrcv x k_w); buffers hold max_windows slots.  Host
 * outputs (max_windows entries): window [lo, hi] (first and last candidate),
 * k, number of expansion points, largest final estimate, and (nullable) how many
 * of the points were reused from enclosing windows.  Errors as rom_greedy. */
fsi_status rom_windows(const fsi_dims* dims, const void* d_model, const fsi_c64* F, int nrhs,
                       const double* cand_hz, int ncand, const fsi_window_opts* opts, void* ws,
                       size_t ws_bytes, const int32_t* rcv, int nrcv, fsi_c64* KR, fsi_c64* DR,
                       fsi_c64* MR, fsi_c64* fR, fsi_c64* CR, int* nwin_out, double* lo_out,
                       double* hi_out, int* k_out, int* nshift_out, double* maxest_out,
                       int* nreused_out, void* stream);

/* Workspace bytes for rom_windows_sweep. */
fsi_status rom_windows_sweep_workspace(int kmax, int nrhs, int batch, size_t* bytes);

/* Reduced sweep with windowed ROMs (layout of rom_windows): every frequency is
 * solved with the window that contains it, else the nearer neighbour.
 * f_hz host, increasing; p_out/spl_out as rom_sweep. */
fsi_status rom_windows_sweep(int nwin, const double* lo, const double* hi, const int* k, int kmax,
                             const fsi_c64* KR, const fsi_c64* DR, const fsi_c64* MR,
                             const fsi_c64* fR, const fsi_c64* CR, int nrhs, int nrcv,
                             const double* f_hz, int nf, int batch, void* ws, size_t ws_bytes,
                             fsi_c64* p_out, double* spl_out, void* stream);

/* One reduced model of a multi-model reduced sweep (all pointers device; the
 * matrices as rom_project writes them: KR/DR/MR k x k, fR k x nrhs, CR nrcv x k,
 * column-major).  k <= 128, nrhs <= 4. */
typedef struct {
    int k, nrhs, nrcv, nf;
    const fsi_c64* KR;
    const fsi_c64* DR;
    const fsi_c64* MR;
    const fsi_c64* fR;
    const fsi_c64* CR;
    const double* f_hz;           /* nf frequencies                                  */
    fsi_c64* p_out;               /* nf x nrcv x nrhs                                */
    double* spl_out;              /* same shape, nullable                            */
} fsi_rom_item;

/* Reduced sweeps (Eq. 11) of nvar models of uneven size in one persistent
 * launch: CTAs take (model, frequency) items, numbered model by model (offsets:
 * device prefix sums of the models' nf, nvar + 1 entries; total = offsets[nvar])
 * from a counter (device int, reset by the call); each item is equilibrated,
 * factored by LU with partial pivoting in FP32 and refined against the FP64
 * residual until the correction is at rounding level (at most 8 steps), then
 * projected to the receivers.  items: device array.
 * Enqueues only a memset and one kernel on the stream (capturable into a CUDA
 * graph); status (device, total, nullable): 0, 1 for a zero or non-finite
 * pivot, 2 for a descriptor out of range, 3 when the refinement did not reach
 * a correction below 1e-12 of the solution (reduced system too ill-conditioned
 * for the FP32 factor: re-solve the item with rom_sweep).  Errors: FSI_EINVAL,
 * FSI_ECUDA. */
fsi_status rom_multi_sweep(const fsi_rom_item* items, int nvar, const int32_t* offsets, int total,
                           int* counter, int32_t* status, void* stream);

/* Learned ROM error estimator (the paper's Sec. 5 suggests a cheaper error
 * estimate than full-order checks; this build learns one).  Network 5 -> 64 ->
 * 64 -> 1, tanh hidden units; parameters flat FP32 [W1 (64x5 row-major), b1,
 * W2 (64x64), b2, W3 (1x64), b3]; forward/backward with FP16-rounded weight
 * matrices and FP32 accumulation. */
#define FSI_MLP_PARAMS 4609

/* Mini-batch Adam (beta 0.9 / 0.999, eps 1e-8) on the mean-squared error of
 * predictions against T, one persistent launch for all steps.  Device arrays:
 * params/adam_m/adam_v (FSI_MLP_PARAMS, updated in place; moments start at 0),
 * X (n x 5 row-major), T (n), order (steps x batch row indices < n), losses
 * (steps, nullable: mean loss of each step's batch), grad_out (FSI_MLP_PARAMS,
 * nullable: gradient of the last step).  step0: steps already taken (bias
 * correction when training resumes).  batch <= 256.  Errors: FSI_EINVAL,
 * FSI_ECUDA. */
fsi_status mlp_train(float* params, float* adam_m, float* adam_v, const float* X, const float* T, int n,
                     const int32_t* order, int steps, int batch, float lr, int step0, float* losses,
                     float* grad_out, void* stream);

/* y[q] = network(X[q]) for q < n (device arrays). */
fsi_status mlp_predict(const float* params, const float* X, int n, float* y, void* stream);

/* Throughput probe for roofline denominators (measurement support; the paper
 * has no counterpart): keeps one execution unit of the current GPU busy with
 * independent operations and no memory traffic, about seconds_hint seconds,
 * timed with CUDA events on `stream`.  kind 0: FP32 FMA (SIMT), 1: FP64 FMA,
 * 2: tcgen05 MMA with BF16 operands, 3: tcgen05 MMA with TF32 operands
 * (M = 128, N = 256, FP32 accumulation), 4: BF16 with M = N = 128 (the
 * tile of the tensor-core LU updates).  scratch: device, >= 1 KiB.  Writes
 * the achieved TFLOP/s (2 flops per multiply-add) and the kernel time in ms.
 * Synchronizes the stream.  Errors: FSI_EINVAL, FSI_ECUDA, FSI_ETIMEOUT. */
fsi_status fsi_probe_peak(int kind, double seconds_hint, void* scratch, double* tflops_out, double* ms_out,
                          void* stream);

const char* fsi_status_str(fsi_status s);
const char* fsi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FSI_H */
