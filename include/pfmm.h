/*
 * pfmm.h -- C ABI of the GB300 (sm_103a) parabolic FMM for the space-time Galerkin boundary
 * element method of the heat equation (arXiv 2106.15911).
 *
 * Problem (Section 2): Dirichlet problem of the heat equation u_t - alpha Laplace u = 0 in
 * Omega x (0, T), zero initial condition, u = g on Gamma x (0, T).  The Neumann datum
 * w = alpha du/dn solves V w = (1/2 I + K) g (Section 2, boundary integral equation).  With a
 * fixed triangulation {gamma_x} of Gamma and E_t uniform steps of length h = T / E_t:
 *
 *   V_h[(k,x),(j,y)] = int_{I_k} int_{gamma_x} int_{I_j} int_{gamma_y} G_alpha(x - y, t - tau)
 *   K_h[(k,x),(j,i)] = same with alpha dG_alpha/dn_y times the p1 hat function phi_i(y)
 *   M_h[(k,x),(k,i)] = int_{I_k} int_{gamma_x} phi_i = h |gamma_x| / 3 for i a vertex of gamma_x
 *
 * (Section 2, the matrix entries after Eq. 02:linear:system.)  V_h and K_h are applied by the
 * space-time FMM of Section 3 (Alg. 2): nearfield blocks (Eq. eval_sl_nf_block) plus S2M
 * (Eq. s2m), M2M (Eq. temp_m2m, st_m2m), M2L (Eq. m2l with Eq. exp_coeffs_3d/1d), L2L and
 * L2T (Eq. l2t) over the box cluster tree of Alg. 1.
 *
 * Vector layouts (all FP64, all DEVICE pointers, caller-owned):
 *   w, f        [nrhs][E_t][E_x]  p0 coefficients, index (k-1) E_x + x of Section 2 per rhs
 *   g           [nrhs][E_t][N_v]  p0-in-time, p1-in-space coefficients (node order of the mesh)
 * Triangles and nodes are in the caller's order; any reordering is internal.
 *
 * Errors: every entry point returns PFMM_OK (0) or a negative code; pfmm_last_error() then
 * returns a message for the calling thread.  No C++ exception crosses this interface.  On an
 * error the output vectors are unspecified.  A handle is not thread-safe: calls on one handle
 * must not overlap (they share the handle's workspaces); different handles are independent.
 */
#ifndef PFMM_H
#define PFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define PFMM_OK 0
#define PFMM_ERR_INVALID_ARG (-1)  /* a pointer is NULL, a size is out of range, ... */
#define PFMM_ERR_OOM (-2)          /* device allocation failed or the memory cap is exceeded */
#define PFMM_ERR_CUDA (-3)         /* a CUDA runtime call or kernel launch failed */
#define PFMM_ERR_NONFINITE (-4)    /* an input holds NaN or Inf */
#define PFMM_ERR_TIMEOUT (-5)      /* a bounded device wait gave up */
#define PFMM_ERR_NOT_CONVERGED (-6)/* the solver stopped before its tolerance */
#define PFMM_ERR_UNSUPPORTED (-7)  /* a valid request this build does not implement */

/* precision modes */
#define PFMM_FP64 0   /* FP64 accuracy in every phase (see pfmm_params.fp64_native for how) */
#define PFMM_MIXED 1  /* FP32 regular-pair quadrature and FP32 FMM passes; FP64 singular
                         quadrature; FP64 output accumulation.  The stored nearfield is applied
                         on the tensor cores (default engine) as three FP16 products of scaled
                         hi/lo parts with FP32 accumulation (about 2^-22 relative, as FP32), or
                         in FP32 on the CUDA cores (PFMM_NF_CUDA_CORES, or where the panel layout
                         does not suit the tensor cores) */

/* nearfield modes */
#define PFMM_NEARFIELD_STORED 0    /* nearfield blocks assembled once at build time */
#define PFMM_NEARFIELD_ONTHEFLY 1  /* blocks recomputed tile by tile inside every apply (only the
                                      Sauter-Schwab values of touching pairs are stored); for
                                      meshes whose blocks do not fit the memory budget */

/* nearfield engines */
#define PFMM_NF_AUTO 0
#define PFMM_NF_CUDA_CORES 1

/* apply parts (bit mask) */
#define PFMM_PART_NEAR 1  /* inadmissible (nearfield) blocks, Alg. 2 last loop */
#define PFMM_PART_FAR 2   /* S2M, M2M, M2L, L2L, L2T, Alg. 2 first four phases */
#define PFMM_PART_ALL 3

/* The tensor space-time mesh (Section 2).  Arrays are HOST pointers, read during
 * pfmm_build_trees only (copied). */
typedef struct pfmm_mesh {
    int32_t n_vertices;      /* N_v */
    int32_t n_triangles;     /* E_x */
    const double *vertices;  /* [N_v][3] */
    const int32_t *triangles;/* [E_x][3] vertex indices, counter-clockwise seen from outside */
    double T;                /* end time */
    int32_t n_steps;         /* E_t, uniform steps h = T / E_t */
    double alpha;            /* heat capacity constant alpha > 0 */
} pfmm_mesh;

/* FMM parameters (Section 3; Alg. 2 line 1 names n_max, c_st, n_tr, m_t, m_x). */
typedef struct pfmm_params {
    int32_t m_t;        /* Lagrange degree in time (Section 3.1), >= 0 */
    int32_t m_x;        /* Chebyshev degree in space (total degree), 0 <= m_x <= 12 */
    double c_st;        /* box-shape constant of Eq. rel_h_t_h_x */
    int32_t n_tr;       /* interaction-area radius of Eq. 03:Iarea; < 0: derived from eps_tr */
    double eps_tr;      /* neglected kernel size when n_tr < 0 */
    int32_t leaf_steps; /* time steps per temporal leaf (E_t / leaf_steps a power of two) */
    int32_t leaf_tris;  /* no spatial refinement once no box holds more triangles */
    int32_t precision;  /* PFMM_FP64 or PFMM_MIXED */
    int32_t nearfield;  /* PFMM_NEARFIELD_STORED (default) or PFMM_NEARFIELD_ONTHEFLY */
    int32_t quad_regular;  /* Gauss points per direction of the collapsed triangle rule */
    int32_t quad_singular; /* Gauss points per direction of the Sauter-Schwab rule */
    int32_t nf_engine;  /* PFMM_NF_AUTO: tensor cores where the panel layout allows (mixed mode: the
                           scaled two-part FP16 split with FP32 accumulation; FP64 mode: exact
                           integer products modulo 16 primes, combined by the Chinese remainder
                           theorem), else CUDA cores; PFMM_NF_CUDA_CORES: always CUDA cores */
    int32_t fp64_native;/* FP64 mode only.  0 (default): FP64-accurate arithmetic on the fast units --
                           the nearfield as exact residue products on the tensor cores (see
                           nf_engine) and the FMM passes in double-FP32 arithmetic (pairs of FP32
                           numbers, about 48 significant bits, on the FP32 pipe); 1: every phase on
                           the FP64 pipe (reference mode, about 50x slower on GB300) */
    int32_t nf_form;    /* FP64 tensor-core nearfield kernel form: 0 (default) the faster of the two,
                           timed at build; 1 one 128-row tile and two moduli per work item; 2 two
                           row tiles sharing each input stage, one modulus per item */
} pfmm_params;

typedef struct pfmm_handle pfmm_handle;

/* Tree statistics of a handle (for tests and logs). */
typedef struct pfmm_info {
    int32_t p;              /* leaf level */
    int32_t lx[32];         /* spatial refinements per level */
    int32_t nbox[32];       /* non-empty spatial boxes per level */
    double pad[32];         /* padding per level */
    int32_t n_m2l_pairs;    /* space-time box pairs in all interaction lists */
    int64_t nearfield_bytes;/* device bytes of the stored nearfield blocks (V and K) */
    int64_t device_bytes;   /* all device bytes held by the handle */
    int32_t nf_tensor_cores;/* bit 0: V nearfield on tensor cores, bit 1: K nearfield */
    int64_t nearfield_v_elements; /* stored V nearfield entries (all panels, all step offsets) */
    int32_t nf_dense_columns;     /* 1: the panels share one column space (all triangles / nodes,
                                     zero where the source is not near), 0: compact per panel */
    int32_t m2l_engine[32];       /* M2L kernel of level l (l = 2 .. p; 0 elsewhere): PFMM_M2L_* */
    int32_t nf_form;              /* form of the FP64 tensor-core nearfield kernel in use (0: none) */
    double nf_form_ms[2];         /* build-time timing of forms 1 and 2 (ms per V product; 0 if not timed) */
    double m2l_flops;             /* flops of one rhs's M2L in the separable form (Eq. m2l with
                                     Eq. exp_coeffs_3d applied one direction at a time over the
                                     full box grid of every level, all interval pairs of Eq.
                                     03:ILtemp and time nodes): 2 x FMAs of the three passes */
} pfmm_info;

/* M2L kernels (pfmm_info.m2l_engine): the three separable passes through a global workspace
 * (FP64, grids beyond 8^3 or high degrees), the fused kernel (FP32, grids of at most 4^3 cells,
 * m_x <= 7), the slab kernel (FP32, grids of 5^3 .. 8^3 cells, m_x <= 6). */
#define PFMM_M2L_THREE_PASS 1
#define PFMM_M2L_FUSED 2
#define PFMM_M2L_SLAB 3
#define PFMM_M2L_FUSED_SLICED 4  /* the fused kernel forming T2 one nu1 at a time (FP32, m_x = 8) */

/* Fill *p with defaults: m_t = 4, m_x = 4, c_st = 1, n_tr = -1, eps_tr = 1e-12,
 * leaf_steps = 2, leaf_tris = 16, FP64, stored nearfield, quad_regular = 3,
 * quad_singular = 6, nf_engine = PFMM_NF_AUTO, fp64_native = 0, nf_form = 0.  Returns PFMM_OK or
 * PFMM_ERR_INVALID_ARG (p NULL). */
int pfmm_default_params(pfmm_params *p);

/* Build the box cluster tree (Section 3.2, Alg. 1), the nearfield and interaction lists
 * (Section 3.3), the expansion tables (Section 3.1, 3.4) and, in stored mode, the nearfield
 * blocks of V_h and K_h (Eq. eval_sl_nf_block).  `stream` is a cudaStream_t (NULL = legacy
 * default stream); the call synchronises it before returning.  On success *out owns device
 * memory until pfmm_destroy. */
int pfmm_build_trees(const pfmm_mesh *mesh, const pfmm_params *params, void *stream, pfmm_handle **out);

/* f = V_h w (Alg. 2), f overwritten.  w, f: device [nrhs][E_t][E_x] FP64, must not overlap.
 * Enqueued on `stream`; returns without synchronising.  nrhs >= 1. */
int pfmm_apply_V(pfmm_handle *h, const double *w, double *f, int32_t nrhs, void *stream);

/* f = K_h g (Alg. 2 with the double-layer moments, Section 3 "slight modifications").
 * g: device [nrhs][E_t][N_v], f: device [nrhs][E_t][E_x], f overwritten. */
int pfmm_apply_K(pfmm_handle *h, const double *g, double *f, int32_t nrhs, void *stream);

/* f = M_h g (p0-p1 mass matrix, Section 2).  g: [nrhs][E_t][N_v], f: [nrhs][E_t][E_x]. */
int pfmm_apply_M(pfmm_handle *h, const double *g, double *f, int32_t nrhs, void *stream);

/* Like pfmm_apply_V / pfmm_apply_K (op 0 / 1) but computing only the parts in `parts`
 * (PFMM_PART_NEAR, PFMM_PART_FAR or both); f is overwritten with that part. */
int pfmm_apply_parts(pfmm_handle *h, int32_t op, const double *x, double *f, int32_t nrhs, int32_t parts,
                     void *stream);

/* Per-phase device times.  When enabled, every apply records CUDA events around its phases on
 * its stream; pfmm_phase_times synchronises the last apply's stream, writes the accumulated
 * milliseconds of the phases (0 permute in, 1 nearfield, 2 S2M, 3 M2M, 4 M2L, 5 L2L, 6 L2T,
 * 7 permute out) and the number of applies measured, then resets the accumulators. */
int pfmm_set_profiling(pfmm_handle *h, int32_t on);
int pfmm_phase_times(pfmm_handle *h, double *ms8, int32_t *n_applies);
/* The nearfield product kernel alone (the tensor-core kernel of the nearfield phase:
 * k_nf_apply_tc in mixed precision, k_nf_apply_crt in FP64 mode), from CUDA events recorded on
 * the apply's stream immediately before and after its launch while profiling is on: the
 * accumulated milliseconds and the number of launches measured since the last call, then reset.
 * Both are 0 when the nearfield ran on the CUDA cores.  Reads the events of the applies that
 * pfmm_phase_times has not yet collected, so call it before pfmm_phase_times. */
int pfmm_nf_kernel_time(pfmm_handle *h, double *ms, int32_t *n_launches);

int pfmm_get_info(const pfmm_handle *h, pfmm_info *info);

/* Measurement utility (not part of the paper's method): the number of kernels one
 * pfmm_apply_parts(h, op, x, f, nrhs, parts) launches.  The apply is captured into a CUDA graph
 * on a private stream (nothing executes; x and f are device buffers of the apply's sizes, not
 * read or written) and its kernel nodes are counted into *kernels.  Sizes the handle's
 * workspaces for nrhs first (may allocate). */
int pfmm_count_apply_kernels(pfmm_handle *h, int32_t op, const double *x, double *f, int32_t nrhs, int32_t parts,
                             int64_t *kernels);

/* Synchronise the device and report whether a bounded wait inside a kernel of this handle gave
 * up since the last check (PFMM_ERR_TIMEOUT; the result of that apply is invalid), or a CUDA
 * error is pending (PFMM_ERR_CUDA).  Clears the flag.  PFMM_OK otherwise. */
int pfmm_check(pfmm_handle *h);

/* Measurement utility (not part of the paper's method): the sustained FMA throughput of the
 * current device in TFLOP/s (2 flops per FMA), FP64 (fp64 != 0) or FP32, timed with CUDA
 * events over five launches of independent FMA chains on `stream`.  Synchronises the stream.
 * The FP32 / FP64 pipe rooflines of the nearfield and M2L kernels are quoted against it. */
int pfmm_probe_fma_rate(int32_t fp64, double *tflops, void *stream);

/* Allocation-free f = V_h w.  The paper has no counterpart: this is a service entry point.
 * pfmm_apply_V sizes its per-call workspaces with cudaMalloc on first use (and again when a
 * larger nrhs arrives); callers that must not allocate device memory while they run -- services
 * for which an allocation mid-run may stall the device or fail with no way to recover, and hosts
 * whose device memory is owned by their own allocator or budget -- use this variant instead.
 * It computes the same product with the same kernels, but takes every workspace from one
 * static device array of 64 MiB (held by each GPU that loads the library until the process
 * exits) and calls no cudaMalloc, cudaFree or allocating library routine.
 *   w, f: device [nrhs][E_t][E_x] FP64 as for pfmm_apply_V (f overwritten).  Returns
 *   PFMM_ERR_OOM with a message naming the bytes needed when the workspaces of this handle and
 *   nrhs do not fit in 64 MiB (the separable-M2L intermediates are processed in chunks that fit).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture.  With lazy module
 * loading (the CUDA runtime's default, CUDA_MODULE_LOADING=LAZY) that first lookup is also when
 * the module holding the array is loaded and its 64 MiB are committed on the device, so make the
 * first call at start-up, while memory is known to be free; if the device has no room then, the
 * call returns PFMM_ERR_OOM.  All calls share the
 * one array: calls whose work overlaps on the GPU (other streams, other threads, other handles)
 * race on it and must be serialised by the caller.  The array keeps the last call's contents;
 * each call writes every workspace before reading it. */
int pfmm_apply_V_noalloc(pfmm_handle *h, const double *w, double *f, int32_t nrhs, void *stream);

/* Representation formula (Section 2): the solution at interior space-time points,
 *   u(x, t) = (V~ w)(x, t) - (W g)(x, t),
 *   V~ w = int_0^t int_Gamma G_alpha(x - y, t - tau) w(y, tau) ds_y dtau,
 *   W g  = int_0^t int_Gamma alpha dG_alpha/dn_y(x - y, t - tau) g(y, tau) ds_y dtau,
 * for the discrete densities of Eq. 02:linear:system: w piecewise constant on the space-time
 * elements (the solution of pfmm_solve, direct formulation) and g piecewise constant in time,
 * piecewise linear in space (the projected Dirichlet datum); with g = NULL only V~ w (the
 * indirect formulation's single-layer ansatz).  The time integrals are exact (first time
 * antiderivatives of the heat kernel); the space integrals use the handle's regular collapsed
 * Gauss rule (quad_regular^2 points per triangle), so points should keep a distance of a few
 * element sizes from Gamma for that rule to be accurate.  Direct summation over all elements in
 * FP64 (no FMM): cost np x E_x x quad_regular^2 x E_t per rhs.
 *   w: device [nrhs][E_t][E_x], g: device [nrhs][E_t][N_v] or NULL, points: device [npoints][4] =
 *   (x, y, z, t) with t > 0 (t <= 0 gives 0; steps beyond E_t do not exist), u: device
 *   [nrhs][npoints] (overwritten).  Enqueued on `stream`; returns without synchronising. */
int pfmm_eval_repr(pfmm_handle *h, const double *w, const double *g, const double *points, int32_t npoints,
                   double *u, int32_t nrhs, void *stream);

/* ---- temporal decomposition over several GPUs (Section 4) ----------------------------------
 * The space-time FMM shards by time: every cluster of the binary temporal tree (levels 0 ..
 * `levels`, 2^l clusters on level l, the leaf intervals on the last level) has one owner rank,
 * which runs the FMM operations of all space-time boxes attached to it.  Owners follow the three
 * rules of Section 4.1 (levels >= ceil(log2 nranks): consecutive ranks in ascending order, as
 * evenly as possible; the level above: the owner of the left child; coarser levels: from each of
 * 2^l consecutive rank groups the rank with the fewest clusters so far).  The messages of one
 * distributed matrix-vector product (Section 4.2) are one-directional per cluster: moments to
 * the owners of the parent (M2M, levels >= 3) and of the M2L targets k + 2 and, for even k, k + 3
 * (Eq. 03:ILtemp, levels >= 2); locals to the owners of the two children (L2L, levels 2 ..
 * levels - 1); the input of a leaf interval to the owner of the next one (nearfield halo).
 * Host logic only (no device work); this build runs one GPU per process and uses it to plan. */
#define PFMM_MSG_MOMENTS 0
#define PFMM_MSG_LOCALS 1
#define PFMM_MSG_INPUT 2
/* owner[(1 << l) - 1 + k] = rank owning cluster k of level l (array of 2^(levels+1) - 1 ints). */
int pfmm_shard_owners(int32_t levels, int32_t nranks, int32_t *owner);
/* The messages as rows (kind, level, interval, source rank, destination rank), in the order of a
 * bottom-up sweep over the levels; at most `cap` rows are written to msgs [cap][5], *count gets
 * the total (call with cap = 0 to size the array). */
int pfmm_shard_messages(int32_t levels, int32_t nranks, int32_t *msgs, int64_t cap, int64_t *count);

/* ---- general (non-uniform) time steps -----------------------------------------------------
 * The space-time FMM of Alg. 2 on the general box cluster tree of Alg. 1 (Section 3.2 in full;
 * the adaptive direction of Section 6): time steps t_0 = 0 < t_1 < ... < t_Et = T of any lengths,
 * boxes refined while they hold at least n_max space-time elements (early leaves on any level),
 * temporal splits at the step nearest an interval's centre, refinement stopped early for oversized
 * elements (an interval of a single step, a step longer than the level's nominal interval length
 * T / 2^l, a triangle wider than its cell), and the nearfield of Eq. def_st_nearfield including
 * the leaves of the ancestors' nearfields (N(parent(Z)) /\ L_Sigma).  No block-Toeplitz
 * structure: the nearfield blocks hold the entries of every (target step, source step) pair.
 * Single layer V_h, FP64.  Vector layouts as above ([nrhs][E_t][E_x], device pointers). */
typedef struct pfmm_gen pfmm_gen;

typedef struct pfmm_gen_info {
    int32_t nlev;            /* levels 0 .. nlev - 1 */
    int32_t lx[32];          /* spatial refinements of level l */
    int32_t nbox[32];        /* boxes of level l */
    int32_t nleaf[32];       /* leaves of level l */
    int32_t nint[32];        /* temporal intervals present on level l */
    int32_t ntr_far[32];     /* interaction-area radius of level l for M2L (Eq. 03:Iarea) */
    int32_t ntr_near[32];    /* ... and for the nearfield */
    int32_t st[32];          /* 1: level l is refined into level l+1 in space and time, 0: in time */
    double pad[32];          /* padding of level l */
    int64_t n_m2l_pairs;     /* box pairs of all interaction lists */
    int64_t n_near_blocks;   /* (leaf, nearfield box) blocks */
    int64_t nearfield_entries; /* stored nearfield entries */
    int64_t device_bytes;    /* device memory held by the handle */
} pfmm_gen_info;

/* Build the general tree, lists, tables and stored nearfield.  mesh: as for pfmm_build_trees with
 * n_steps = E_t and T = t_steps[E_t]; t_steps: HOST array of E_t + 1 times, t_steps[0] = 0,
 * strictly increasing (copied).  params: m_t, m_x, c_st, n_tr, eps_tr, quad_regular and
 * quad_singular are used (leaf_steps, leaf_tris, nearfield, nf_engine, fp64_native and nf_form
 * are ignored; precision must be PFMM_FP64, else PFMM_ERR_UNSUPPORTED).  n_max >= 1: the element
 * bound of Alg. 1.  Returns PFMM_ERR_OOM when the stored nearfield exceeds 60 % of the free device
 * memory.  Synchronises `stream`. */
int pfmm_gen_create(const pfmm_mesh *mesh, const double *t_steps, const pfmm_params *params, int32_t n_max,
                    void *stream, pfmm_gen **out);
/* f = V_h w (Alg. 2, parts as for pfmm_apply_parts), f overwritten; w, f device [nrhs][E_t][E_x]
 * FP64, must not overlap.  Enqueued on `stream`; may allocate workspaces on first use or a larger
 * nrhs. */
int pfmm_gen_apply_V(pfmm_gen *h, const double *w, double *f, int32_t nrhs, int32_t parts, void *stream);
int pfmm_gen_get_info(const pfmm_gen *h, pfmm_gen_info *info);
/* The boxes as rows (level, cell x, cell y, cell z, interval k, leaf, first step, end step), level
 * by level; at most cap rows into rows [cap][8], *count gets the total. */
int pfmm_gen_boxes(const pfmm_gen *h, int32_t *rows, int64_t cap, int64_t *count);
void pfmm_gen_destroy(pfmm_gen *h);

/* ---- solver ------------------------------------------------------------------------------ */
#define PFMM_DIRECT 0    /* V_h w = (1/2 M_h + K_h) g  (Section 2, Eq. 02:linear:system) */
#define PFMM_INDIRECT 1  /* V_h w = M_h g              (single-layer ansatz) */

typedef struct pfmm_mpnn pfmm_mpnn;  /* learned preconditioner (see the end of this header) */

typedef struct pfmm_solve_opts {
    double tol;           /* stop when ||b - V_h x||_2 <= tol ||b||_2 (default 1e-8) */
    int32_t restart;      /* FGMRES restart length m (default 50, at most 500) */
    int32_t max_it;       /* cap on inner iterations (V_h applies of the inner handle), default 1000 */
    pfmm_handle *refine;  /* optional FP64 handle of the same problem: GMRES-IR (default NULL) */
    double inner_tol;     /* GMRES-IR: relative tolerance of each inner solve (default 1e-4) */
    int32_t max_outer;    /* GMRES-IR: cap on refinement steps (default 20) */
    pfmm_mpnn *precond;   /* optional learned right preconditioner z = P(v); NULL: identity */
    double *rec_r;        /* optional device [rec_cap][E_t][E_x]: recorded residuals r_k = b - V x_k */
    double *rec_e;        /* optional (nullable) device [rec_cap][E_t][E_x]: errors e_k = x - x_k */
    int32_t rec_cap;      /* number of (r, e) slots (0: no recording; needs refine == NULL) */
    int32_t rec_every;    /* record at every rec_every-th Arnoldi step of each cycle (default 5) */
    int32_t rec_basis;    /* 1: record the Arnoldi basis vectors v_j into rec_r instead (rec_e unused) */
} pfmm_solve_opts;

typedef struct pfmm_solve_info {
    int32_t iterations;   /* inner FGMRES iterations over all right-hand sides */
    int32_t outer;        /* refinement steps (GMRES-IR) */
    double rel_res;       /* largest final ||b - V_h x|| / ||b|| (FP64 operator when refining) */
    double seconds;       /* wall time of the call */
    int32_t recorded;     /* (r, e) pairs written to rec_r / rec_e */
    int32_t precond_off;  /* cycles after which the preconditioner was dropped (non-finite output
                           * or a cycle that cut the residual by less than 10 %) */
} pfmm_solve_info;

int pfmm_default_solve_opts(pfmm_solve_opts *opts);

/* Solve V_h x = b for every right-hand side, b = (1/2 M_h + K_h) g (PFMM_DIRECT) or M_h g
 * (PFMM_INDIRECT), with restarted right-preconditioned flexible GMRES (x0 = 0, Arnoldi by
 * classical Gram-Schmidt applied twice), all Krylov vectors FP64 on the device.  With
 * opts->refine (an FP64 handle of the same mesh and steps) the residual is formed in FP64 with
 * it and inner FGMRES solves run with h (typically PFMM_MIXED): iterative refinement.
 * With opts->precond the Krylov directions are z_j = P(v_j) (flexible GMRES, so P may be
 * nonlinear); the residuals are still those of the exact operator, and P is dropped for the rest
 * of the solve when it yields a non-finite vector or a cycle that cuts the residual by < 10 %.
 * Recording (rec_cap > 0, plain FGMRES only): at Arnoldi steps j = 0, rec_every, 2 rec_every ...
 * of every cycle, while the residual is above 100 tol ||b||, the iterate x_j and its residual
 * r_j = b - V_h x_j (from the Arnoldi relation) are kept; after convergence rec_e holds x - x_j:
 * the (residual, error) pairs a preconditioner is trained on.
 *   g: device [nrhs][E_t][N_v] (p0 in time, p1 in space, already projected), x: device
 *   [nrhs][E_t][E_x] (overwritten).  Synchronises `stream`; allocates its Krylov workspace
 *   ((2 restart + 4) E_t E_x doubles).  Returns PFMM_ERR_NOT_CONVERGED when a cap is reached
 *   (x holds the last iterate and info is filled), PFMM_ERR_NONFINITE for NaN / Inf in g. */
int pfmm_solve(pfmm_handle *h, int32_t formulation, const double *g, double *x, int32_t nrhs,
               const pfmm_solve_opts *opts, pfmm_solve_info *info, void *stream);

/* ---- batches of independent problems ------------------------------------------------------ */
typedef struct pfmm_batch pfmm_batch;

/* Choose the spatial degree m_x in [m_lo, m_hi] for a problem a priori: the smallest degree
 * whose first dropped Chebyshev coefficient of the Gaussian factor (Eq. exp_coeffs_1d, at the
 * smallest d_ab over the M2L levels of the problem's tree) is below tol times the leading one.
 * *out = *base with m_x replaced.  Host only. */
int pfmm_autotune_params(const pfmm_mesh *mesh, const pfmm_params *base, double tol, int32_t m_lo, int32_t m_hi,
                         pfmm_params *out);

/* Build n independent problems (one handle each, own tree, tables and nearfield).  With
 * tune_engines != 0, per problem and timed with CUDA events: the tensor-core and CUDA-core
 * nearfield applies (where the panels allow the tensor cores), and the M2L kernel forms (the
 * per-level default, the fused kernel, its sliced form, the three global passes, each where it can
 * run the problem's levels) on the far field; the fastest of each is kept (pfmm_get_info reports
 * the resulting M2L engine per level).  Synchronises `stream`. */
int pfmm_build_trees_batched(int32_t n, const pfmm_mesh *meshes, const pfmm_params *params, int32_t tune_engines,
                             void *stream, pfmm_batch **out);

/* f[i] = V_h(i) w[i] for all problems i of the batch (device pointers, layouts as for
 * pfmm_apply_V, nrhs[i] right-hand sides each).  The first call (and any call with different
 * pointers or counts) sizes the workspaces and captures the whole batch into one CUDA graph, one
 * branch per problem on a pool of up to 16 streams; later calls replay it on `stream`. */
int pfmm_apply_V_batched(pfmm_batch *b, const double *const *w, double *const *f, const int32_t *nrhs,
                         void *stream);

int pfmm_batch_handle(pfmm_batch *b, int32_t i, pfmm_handle **h);  /* the i-th problem's handle */
int32_t pfmm_batch_size(const pfmm_batch *b);
/* Branches of the captured graph run on a pool of nstreams streams (default min(n, 16)); the
 * next pfmm_apply_V_batched captures again. */
int pfmm_batch_set_streams(pfmm_batch *b, int32_t nstreams);
void pfmm_batch_destroy(pfmm_batch *b);

/* ---- learned preconditioner ---------------------------------------------------------------
 * The paper has no counterpart (it solves with unpreconditioned GMRES).  A message-passing
 * network over the triangle edge adjacency acts on each time slice v_t ([E_x] values) of a vector:
 *   f_i = (|gamma_i| / mean area, outward unit normal n_i, (t + 1/2) / E_t),  s_t = RMS(v_t) + 1e-30,
 *   e_i = SiLU(W_g^T f_i + b_g),  h^0_i = (v_i / s_t) e_i,
 *   h^{l+1} = h^l + W_s^T h^l + W_n^T mean_{j ~ i} h^l_j  (l < layers),
 *   z_i = c s_t (w_o . h^L_i),  j ~ i: triangles sharing an edge with i.
 * z is linear in v (FGMRES needs a consistent preconditioner); the coefficients depend on the
 * geometry through e.  Weights are used in BF16 (FP32 master copies for Adam), accumulation is
 * FP32.  Parameters (FP32, this order, matrices input-major M[k][o]): W_g [5][W], b_g [W], per
 * layer {W_s [W][W], W_n [W][W]}, w_o [W].  Training data are residual slices r_b recorded by
 * pfmm_solve (with their errors e_b, V_h e = r).  Two losses over a batch of S slices:
 *   same-step form (a pFMM handle h of the mesh given): the correction wanted for r_b is
 *     c_b = A_0^{-1} r_b, A_0 the same-step (time-block-diagonal) nearfield block of V_h, measured
 *     in the residual norm:  (1/S) sum_b ||A_0 z(r_b) - r_b||^2 / (||r_b||^2 + 1e-30);
 *     the gradient uses A_0 for A_0^T (symmetric up to the singular quadrature error);
 *   error form (h NULL):  (1/S) sum_b ||z(r_b) - e_b||^2 / (||e_b||^2 + 1e-30). */

/* Network for a mesh (host arrays copied; E_t = mesh->n_steps).  width: 16, 32 or 64; layers
 * 0..16; weights drawn from `seed`.  The output scale c is unset (0) until set or estimated by
 * the first pfmm_mpnn_train call. */
int pfmm_mpnn_create(const pfmm_mesh *mesh, int32_t width, int32_t layers, uint64_t seed, pfmm_mpnn **out);
int64_t pfmm_mpnn_num_params(const pfmm_mpnn *net);
/* FP32 master parameters to / from host memory (n = pfmm_mpnn_num_params); set resets Adam. */
int pfmm_mpnn_get_params(const pfmm_mpnn *net, float *host, int64_t n);
int pfmm_mpnn_set_params(pfmm_mpnn *net, const float *host, int64_t n);
int pfmm_mpnn_set_output_scale(pfmm_mpnn *net, float c);
int pfmm_mpnn_get_output_scale(const pfmm_mpnn *net, float *c);
/* z = P(v) for nvec vectors, v and z device [nvec][E_t][E_x] FP64 (z overwritten). */
int pfmm_mpnn_apply(pfmm_mpnn *net, const double *v, double *z, int32_t nvec, void *stream);
/* Loss and gradient w.r.t. the parameters for the slices slices[0..n) (host array of indices
 * s into the device arrays R, E of [*][E_t][E_x] FP64: slice s holds elements s E_x .. s E_x +
 * E_x - 1 and has step s mod E_t; the caller guarantees s < the arrays' slice count).  h: a
 * handle of the same mesh and E_t for the same-step form, NULL for the error form (then E is
 * required; otherwise it may be NULL).  loss / grad (host, nullable) receive the values; no
 * parameter update.  Synchronises `stream`. */
int pfmm_mpnn_loss_grad(pfmm_mpnn *net, pfmm_handle *h, const double *R, const double *E, const int32_t *slices,
                        int32_t nslices, float *loss, float *grad, void *stream);
/* `steps` Adam steps on batches of batch_slices slices drawn uniformly (generator seeded by
 * `seed`) from the nvec recorded vectors R (and E), device [nvec][E_t][E_x] FP64, with the loss
 * form chosen by h as for pfmm_mpnn_loss_grad; step size lr, cosine-decayed to lr / 10.  An unset
 * output scale is first estimated from one batch.  loss_history (host, nullable) receives each
 * step's loss.  Synchronises `stream`. */
int pfmm_mpnn_train(pfmm_mpnn *net, pfmm_handle *h, const double *R, const double *E, int64_t nvec, int32_t steps,
                    int32_t batch_slices, float lr, uint64_t seed, float *loss_history, void *stream);
/* Compiled form: the network is linear in each slice and each layer reaches one more edge
 * neighbour, so for every step t it equals a sparse operator P_t whose row i lives on the ball
 * of `layers` edges around triangle i.  This assembles P_t (FP32) by probing: the triangles are
 * coloured so that any two within 2 layers edges differ, the network is applied (with its own
 * kernels) to one 0/1 probe per colour, and each result fills the ball entries of that colour.
 * Afterwards pfmm_mpnn_apply computes z = P_t v (FP32 input copy and sums, FP64 output); any
 * parameter change (set_params,
 * training, set_output_scale) drops the compiled form.  Needs E_t * E_x * max ball size floats.
 * Synchronises `stream`. */
int pfmm_mpnn_compile(pfmm_mpnn *net, void *stream);
/* Reads and clears the network's error word: PFMM_ERR_TIMEOUT when a bounded wait of its
 * tensor-core kernels gave up since the last check (pfmm_mpnn_apply is asynchronous; training
 * and pfmm_solve check on return).  Synchronises the device. */
int pfmm_mpnn_check(pfmm_mpnn *net);
void pfmm_mpnn_destroy(pfmm_mpnn *net);

/* Release the handle and its device memory (NULL is ignored). */
void pfmm_destroy(pfmm_handle *h);

/* Message of the last error on the calling thread ("" if none). */
const char *pfmm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PFMM_H */
