/*
 * ccmg.h - C ABI of the GB300 cut-cell multigrid library.
 *
 * The library solves  a u_xx + b u_xy + c u_yy = f  (b^2 < 4ac) on a square
 * box minus a union of holes (ellipses, a flower-shaped polar curve, or the
 * outside of a rotated rectangle), with Dirichlet, Neumann or Robin data
 * N u = g on every boundary curve (Sec. 1, Eq. 1.1-1.2), by the fourth-order
 * cut-cell finite-volume discretisation (Sec. 3-4) and the cut-cell geometric
 * multigrid solver (Sec. 5).  The unknowns are cell averages <u>_i over the
 * cut cells of an N x N Cartesian grid (Eq. 4.1).
 *
 * Conventions shared by every entry point
 *  - Grid vectors are N x N row-major arrays of doubles, index j*N + i, i the
 *    x index (fastest), j the y index; cell (i,j) covers
 *    [x0 + i h, x0 + (i+1) h] x [y0 + j h, y0 + (j+1) h], h = (x1 - x0)/N.
 *    Entries of empty control volumes (outside the domain or merged into a
 *    neighbour by Alg. 1) are ignored on input and written as 0.
 *  - The boundary-data vector g has 4 N + n_bd entries: the face averages of
 *    N u on the south (y = y0, by i), east (x = x1, by j), north (y = y1, by
 *    i) and west (x = x0, by j) box faces, then one boundary average
 *    <<N u>>_i (Eq. 4.2) per cut cell that touches a hole, in row-major cell
 *    order (cc_query reports n_bd; cc_quadrature_nodes gives their rules in
 *    that order).  Entries of
 *    faces that are not used by the discretisation are ignored.
 *  - Pointers named d_* are device pointers on the device that was current
 *    at cc_setup; h_* are host pointers.  The caller owns every array passed
 *    in; the library owns the handle and everything it allocates.
 *  - Every call returns a cc_status; no call throws or aborts.  A call that
 *    fails leaves its outputs unspecified and the handle usable.
 *  - Device work is issued on the stream argument (0 = legacy default) and
 *    is stream-ordered; calls that return host data synchronise that stream.
 *  - A handle may be used from one host thread at a time, except
 *    cc_submit / cc_poll, which are thread-safe.
 */
#ifndef CCMG_H
#define CCMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_hierarchy* cc_handle;
typedef void* cc_stream;            /* a cudaStream_t */

typedef enum {
  CC_OK = 0,
  CC_ERR_ARG = 1,             /* invalid argument (null pointer, bad size, b^2 >= 4ac, ...) */
  CC_ERR_GEOMETRY = 2,        /* the finest grid does not resolve the domain (Alg. 1 precondition) */
  CC_ERR_SINGULAR = 3,        /* a PLG fit, a block factorisation or the bottom matrix is singular */
  CC_ERR_NO_MEMORY = 4,       /* a device or host allocation failed */
  CC_ERR_NOT_CONVERGED = 5,   /* max_cycles reached above the tolerance */
  CC_ERR_DIVERGED = 6,        /* the residual grew by more than 1e3 or became non-finite */
  CC_ERR_TIMEOUT = 7,         /* a bounded wait expired */
  CC_ERR_CUDA = 8,            /* a CUDA runtime call failed */
  CC_ERR_BUSY = 9             /* the request is still in flight (cc_poll) */
} cc_status;

enum { CC_HOLE_ELLIPSE = 0, CC_HOLE_FLOWER = 1, CC_HOLE_OUTSIDE_RECT = 2 };
enum { CC_BC_DIRICHLET = 0, CC_BC_NEUMANN = 1, CC_BC_ROBIN = 2 };
enum { CC_CYCLE_V = 1, CC_CYCLE_W = 2, CC_CYCLE_FMG = 3 };
enum { CC_PREC_FP64 = 0, CC_PREC_MIXED = 1 };
enum { CC_SMOOTHER_JACOBI = 0, CC_SMOOTHER_MCGS = 1 };

/* A hole.  kind CC_HOLE_ELLIPSE: centre (cx, cy), semi-axes r1, r2, rotation
 * theta (rad).  kind CC_HOLE_FLOWER (Sec. 6.2): the region
 * r <= r1 + r2 cos(theta * phi) in polar coordinates (r, phi) about (cx, cy),
 * with 0 < r2 < r1 and theta the number of petals (an integer >= 1).
 * kind CC_HOLE_OUTSIDE_RECT: everything outside the rectangle with corner
 * (cx, cy) and sides r1 (direction theta) and r2 (direction theta + pi/2),
 * so that the domain is that rectangle (Sec. 6.1, the rotated square); it
 * must lie inside the box and be the only hole. */
typedef struct { int kind; double cx, cy, r1, r2, theta; } cc_hole;

/* The domain: the square [x0,x1] x [y0,y1] minus the union of the holes.
 * Holes may overlap one another but must stay inside the box. */
typedef struct { double x0, y0, x1, y1; int n_holes; const cc_hole* holes; } cc_domain;

/* A boundary condition N u = g: Dirichlet (u), Neumann (du/dn, n the outward
 * normal of the domain) or Robin (alpha1 u + alpha2 du/dn). */
typedef struct { int type; double alpha1, alpha2; } cc_bc;

/* Options; cc_default_options fills the defaults noted below. */
typedef struct {
  double eps;          /* Alg. 1 volume-fraction threshold (0.1) */
  int nu1, nu2;        /* pre/post smoothing sweeps (3, 3) */
  double omega;        /* Jacobi weight of the block smoother (0.5) */
  int cycle;           /* CC_CYCLE_V / W / FMG (CC_CYCLE_V) */
  int min_coarse_n;    /* coarsest level: smallest N >= this reached by halving while
                          every hole stays two cells across (4) */
  int precision;       /* CC_PREC_FP64 or CC_PREC_MIXED (FP64) */
  int max_cycles;      /* cycle limit of cc_solve (100) */
  int use_graphs;      /* capture one cycle in a CUDA graph and replay it (1) */
  int host_only;       /* build the tables on the host only, no device work (0);
                          such a handle answers cc_query, cc_cell_types,
                          cc_quadrature_nodes and cc_level_tables only */
  int fmg_cycle;       /* with cycle = CC_CYCLE_FMG: the cycle Alg. 3 runs on each
                          level, CC_CYCLE_V (the paper's, default) or CC_CYCLE_W */
  int w_depth;         /* W cycles: only the w_depth finest levels repeat their
                          coarse-grid correction; coarser levels recurse once.
                          0 (default): every level, the plain W-cycle.  With 1
                          the cycle converges like the W-cycle on the domains
                          tested while each coarse level is visited twice per
                          cycle instead of 2^l times */
  int serve_slots;     /* cc_submit: requests of this handle in flight at once (4);
                          the slots beyond the first are clones (cc_clone) made
                          when needed, within the cc_serve_budget cap */
  int cache;           /* 1: reuse the setup of an identical earlier cc_setup call
                          of this process (same domain, coefficients, conditions,
                          N, eps, omega, min_coarse_n, hole_cells): the handle is
                          then a clone of that hierarchy and setup costs no host
                          time (0) */
  double hole_cells;   /* a coarse level must resolve every hole by this many cells
                          across its smaller semi-axis (2.0).  With holes of 2-5
                          coarse cells some cut-cell rows of the coarsest level can
                          get a diagonal of the wrong sign, and the cycle alone then
                          diverges (see krylov).  A larger value makes the coarsest
                          level finer (setup rejects one above 4096 unknowns with
                          CC_ERR_ARG) */
  int krylov;          /* 0 (default): the solve iterates the cycle (Alg. 2, inside
                          FP64 refinement in the mixed mode).  k in 1..32: restarted
                          flexible GMRES(k) in FP64 on A u = b instead, each step
                          preconditioned by one cycle from zero in the handle's
                          precision, so solves can converge where the cycle alone
                          diverges.  Not part of the paper's method.  Cycle V or W
                          only; cc_result.cycles then counts preconditioner cycles.
                          Where the cycle amplifies some error modes by ~1e6 an FP32
                          cycle keeps too few digits of the rest: use CC_PREC_FP64
                          there.  The handle holds 2k + 4 extra FP64 vectors of the
                          finest grid */
  int smoother;        /* CC_SMOOTHER_JACOBI (default): the block smoother of Def. 5.6,
                          weighted Jacobi on the SFV cells, then the exact block solve.
                          CC_SMOOTHER_MCGS: a variant outside the paper, the SFV cells
                          relaxed colour class by colour class with the latest values
                          of the others (4 classes (i + j) mod 4 for b = 0, 15 classes
                          (i + 4 j) mod 15 otherwise, one in-place launch each), then
                          the same exact block solve; omega 0.6 suits it (the
                          two-grid rate of 2 + 2 sweeps is then about that of the
                          Jacobi smoother's 3 + 3), and omega 1 diverges on this
                          fourth-order stencil */
  int device_setup;    /* 1 (default): the per-cell steps of the setup run as FP64
                          CUDA kernels, one thread per cell: the classification of
                          the cells no curve crosses (Sec. 3.1), the kinds of Def.
                          4.1, the poised lattices (Def. 4.3), the fits (Eq. 4.14,
                          4.17-4.18) and the curve-order samples of Def. 5.1; the
                          tables are bitwise those of the host path.  0: the same
                          steps on host threads.  Ignored with host_only */
  int device_loop;     /* 1 (default): the iterations of a cc_solve or cc_solve_host
                          run inside one CUDA graph launch: a conditional WHILE node
                          repeats the iteration (cycle and FP64 residual) while a
                          one-thread kernel finds the relative residual above tol, so
                          the host waits once per solve; same results as 0.  0: the
                          host reads the residual after every iteration.  The host
                          loop is also used with use_graphs = 0, krylov, cc_kernel_timing
                          on, and for cc_solve_batch and cc_submit, where concurrent
                          solves overlap better under it */
  int autotune;        /* 1 (default): cc_setup times candidate launch shapes on the
                          device and keeps the fastest: the CTA count of the streamed
                          FP32 sweep of each level of 256^2 and more (every multiple of
                          the SM count up to the occupancy limit, and one CTA per tile;
                          the sweep's result does not depend on it), remembered per
                          device and grid size for the process; and the chunk size of
                          each chunked exact block of up to 8192 cells, among the three
                          cheapest by the shared-memory cost model that solve to
                          rounding accuracy (20 timed FP32 solves each).  0: the cost
                          model's choices */
} cc_options;

/* Sizes of a hierarchy. */
typedef struct {
  int n;               /* cells per side on the finest level */
  int n_levels;        /* levels, finest first */
  int64_t n_dof;       /* non-empty cells on the finest level */
  int n_bd;            /* boundary cells (tail of g) */
  int n_g;             /* 4 n + n_bd */
  int n_plg;           /* PLG cells on the finest level */
  int n_block;         /* cells solved exactly by the block smoother, finest level */
  int64_t device_bytes;/* device memory held by the handle */
  int level_n[32];     /* cells per side of each level */
  double block_error;  /* largest normwise backward error of the exact block solves, measured
                          at setup on a fixed vector: |A x - t|_inf / (|A|_inf |x|_inf) */
  double bottom_error; /* the same for the coarsest-level solve */
  int block_m[32];     /* cells of each level's exactly solved block (Eq. 5.8) */
  int block_chunks[32];/* how that block is solved: 0 with its dense inverse in one launch
                          (up to 1024 cells), else the number of chunks of the two-launch
                          chunked form (one CTA per chunk) */
  double setup_seconds;   /* wall time of the cc_setup call that built the tables
                             (0 for a clone or a cached setup) */
  double setup_tables_seconds; /* of which the per-level tables of Sec. 3-4: cut cells,
                             merging, kinds, lattices, fits, block order and rows (the
                             rest: the factorisations of the block smoother and the
                             bottom solve, and the uploads) */
  double setup_kernel_ms; /* device time of the setup kernels (device_setup) */
  int sweep_ctas[32];     /* CTAs of each level's streamed FP32 sweep (0: not streamed) */
  int block_chunk_rows[32]; /* rows per chunk of each chunked exact block (0: dense or none) */
} cc_info;

/* Outcome of a solve. */
typedef struct {
  cc_status status;
  int cycles;          /* cycles (or refinement steps) performed */
  double rel_res;      /* final ||b - A u||_inf / ||b||_inf, FP64 */
  double t_submit, t_start, t_done;   /* seconds, cc_submit/cc_poll only */
  int64_t kernels;     /* CUDA kernels the call launched (graph nodes count once per replay) */
} cc_result;

/* Fill *opt with the defaults. */
void cc_default_options(cc_options* opt);

/* Human-readable name of a status. */
const char* cc_status_string(cc_status s);

/* Text of the last error that made a call from this host thread return
 * CC_ERR_CUDA or CC_ERR_NO_MEMORY, of the setup step that made cc_setup
 * reject a problem (e.g. "singular PLG fit" with CC_ERR_SINGULAR), or of
 * a size limit that made cc_smooth_noalloc return CC_ERR_ARG ("" if none);
 * valid until the next call that sets it. */
const char* cc_last_error_string(void);

/*
 * cc_setup: build the multigrid hierarchy (Sec. 3-5, Eq. 5.9) in FP64 on the
 * host and upload its per-level tables to the current device.
 *   dom      domain; the box must be square and is divided into n x n cells
 *   a, b, c  operator coefficients, b^2 < 4ac
 *   bc       n_bc conditions: bc[0..3] for the south, east, north, west box
 *            sides, bc[4 + k] for hole k (overlapping holes should share one)
 *   n        cells per side of the finest level (even down to the coarsest)
 *   opt      options or NULL for the defaults
 *   stream   stream for the uploads
 *   out      receives the handle; release it with cc_destroy
 * Errors: CC_ERR_ARG, CC_ERR_GEOMETRY (finest level unresolved),
 * CC_ERR_SINGULAR (no poised lattice or a singular block), CC_ERR_NO_MEMORY,
 * CC_ERR_CUDA.  On error *out is NULL.
 */
cc_status cc_setup(const cc_domain* dom, double a, double b, double c,
                   const cc_bc* bc, int n_bc, int n, const cc_options* opt,
                   cc_stream stream, cc_handle* out);

/* Sizes of the hierarchy (host call, no device work). */
cc_status cc_query(cc_handle h, cc_info* out);

/* Release a handle and all its device memory (synchronises the device). */
cc_status cc_destroy(cc_handle h);

/*
 * cc_cell_types: copy the finest-level cell classification to host memory.
 *   h_type[N*N]: 0 empty, 1 full (regular) cell, 2 cut (irregular) cell.
 *   h_kind[N*N] (may be NULL): 0 empty, 1 SFV cell, 2 PLG cell (Def. 4.1).
 *   h_vol[N*N] (may be NULL): cell volumes.
 */
cc_status cc_cell_types(cc_handle h, uint8_t* h_type, uint8_t* h_kind, double* h_vol);

/*
 * cc_quadrature_nodes: quadrature rules on the finest level's cut cells, so
 * that a caller can form the inputs f (Eq. 4.1) and g (Eq. 4.2) there.
 * Call once with NULL arrays to get the counts, then with arrays that size.
 *   n_cut     number of cut cells; h_cell[n_cut] their row-major indices
 *   h_vptr[n_cut+1], h_vnode[3*nv]: volume rule of cell k is nodes
 *             vptr[k] .. vptr[k+1]-1 with (x, y, w), sum of w = 1
 *   h_bptr[n_bd+1], h_bnode[5*nb], h_bbc[nb]: boundary rule of boundary cell
 *             r (same order as the tail of g): (x, y, nx, ny, w) with the
 *             outward normal of the domain, sum of w = 1, and the index of the
 *             condition (into the bc array of cc_setup) that applies there.
 */
cc_status cc_quadrature_nodes(cc_handle h, int* n_cut, int64_t* nv, int64_t* nb,
                              int* h_cell, int64_t* h_vptr, double* h_vnode,
                              int64_t* h_bptr, double* h_bnode, int* h_bbc);

/*
 * cc_solve: solve A u = f - N g (Eq. 4.20) to ||b - A u||_inf / ||b||_inf
 * < tol (FP64 residual), with the method chosen at setup: repeated cycles of
 * Alg. 2 (V or W) or Alg. 3 (FMG) on u in FP64, or, in the mixed precision
 * mode, FP32 cycles on the residual equation inside an FP64 refinement loop.
 *   d_f[N*N]  cell averages of f;  d_g[n_g] boundary data;  d_u[N*N] the
 *   initial guess on input, the solution on output.  All device pointers.
 *   out (may be NULL) receives cycles and the final relative residual.
 * Errors: CC_ERR_ARG, CC_ERR_NOT_CONVERGED, CC_ERR_DIVERGED, CC_ERR_CUDA.
 */
cc_status cc_solve(cc_handle h, const double* d_f, const double* d_g, double* d_u,
                   double tol, cc_stream stream, cc_result* out);

/*
 * cc_clone: a second handle on the hierarchy of src.  It shares every
 * read-only device table of src (class maps, stencil data, block inverses,
 * the coarsest-level inverse) and the host-side setup, and owns its work
 * arrays, CUDA graphs, norm buffer and stream, so that solves on src and on
 * its clones can run at the same time (cc_solve_batch, or cc_solve from
 * different host threads).  No setup is repeated: a clone costs the work
 * arrays only (about 2 x 12 bytes per cell over all levels).  The shared
 * tables stay allocated until src and all its clones are destroyed; destroy
 * each with cc_destroy.  The current device must be src's device.
 * Errors: CC_ERR_ARG (NULL, host-only or wrong device), CC_ERR_NO_MEMORY,
 * CC_ERR_CUDA.  The paper's method needs no counterpart of this call.
 */
cc_status cc_clone(cc_handle src, cc_stream stream, cc_handle* out);

/*
 * cc_solve_batch: n independent solves at once, solve i as cc_solve on
 * handle h[i] with d_f[i], d_g[i], d_u[i] and tolerance tol[i].  The handles
 * must be distinct (clones of one hierarchy are; a handle twice is
 * CC_ERR_ARG).  Solve i runs on streams[i], or, with streams NULL, on h[i]'s
 * own stream after a device synchronisation (so inputs written by earlier
 * work on any stream are visible).  One host thread advances every solve as
 * soon as its previous step has completed on the GPU, so the solves' kernels
 * overlap on the device.  Each solve does exactly the arithmetic of cc_solve
 * on its handle.  out[i] (out may be NULL) receives solve i's result; the
 * return value is CC_OK if every solve converged, else the first failing
 * status.  Outputs are complete on return.
 */
cc_status cc_solve_batch(int n, const cc_handle* h, const double* const* d_f,
                         const double* const* d_g, double* const* d_u, const double* tol,
                         const cc_stream* streams, cc_result* out);

/*
 * cc_solve_host: cc_solve with host arrays h_f, h_g, h_u (same layouts).  The
 * library copies them to and from device buffers that the handle owns; the
 * call returns after the solution is back in h_u.
 */
cc_status cc_solve_host(cc_handle h, const double* h_f, const double* h_g, double* h_u,
                        double tol, cc_stream stream, cc_result* out);

/*
 * cc_submit / cc_poll: streamed requests with continuous batching.
 * cc_submit queues a solve of (d_f, d_g) into d_u on the handle and returns at
 * once with a request id; the arrays must be ready (their producers finished)
 * when cc_submit is called and must stay valid until cc_poll reports
 * completion.  A scheduler thread of the handle admits queued requests in
 * order whenever one of its serve_slots slots is free (the handle itself, or
 * a clone made on demand within the cc_serve_budget cap) and advances every
 * request in flight as soon as its previous step has completed on the GPU,
 * so requests that arrive while others run overlap with them on the device.
 * Each request does exactly the arithmetic of cc_solve.  Do not call cc_solve
 * on a handle while it serves requests.  cc_poll returns CC_ERR_BUSY while
 * the request is queued or running, else the request's final status with its
 * result in *out (timestamps are seconds on a monotonic host clock: submit,
 * admission to a slot, completion).  A finished request is forgotten after
 * the first poll that reports it.
 */
cc_status cc_submit(cc_handle h, const double* d_f, const double* d_g, double* d_u,
                    double tol, uint64_t* req_id);
cc_status cc_poll(uint64_t req_id, cc_result* out);

/*
 * cc_cache_clear: destroy the hierarchies held by the setup cache
 * (cc_options.cache).  Handles made from them stay valid: they keep the
 * shared tables alive until they are destroyed.
 */
cc_status cc_cache_clear(void);

/*
 * cc_serve_budget: cap, in bytes, on the device memory that the serving
 * clones of all handles of this process may hold together (0: no cap, the
 * default).  A scheduler whose next clone would pass the cap keeps requests
 * queued until one of its slots frees.  Errors: CC_ERR_ARG for bytes < 0.
 */
cc_status cc_serve_budget(int64_t bytes);

/* ---- operator-level entry points (one step of the method each) ------------
 * All take FP64 device arrays of the named level's size N_l x N_l and run on
 * `stream`.  They exist so that each step can be checked on its own.
 */

/* b = f - N g on the finest level (Eq. 4.20). */
cc_status cc_assemble_rhs(cc_handle h, const double* d_f, const double* d_g, double* d_b,
                          cc_stream stream);
/* r = b - A u on level l (Eq. 4.23), every non-empty cell. */
cc_status cc_residual(cc_handle h, int level, const double* d_u, const double* d_b,
                      double* d_r, cc_stream stream);
/* One sweep of the block smoother T_omega (Def. 5.6) on level l, u in place. */
cc_status cc_smooth(cc_handle h, int level, double* d_u, const double* d_b, cc_stream stream);
/* r_c = restriction (Eq. 5.10) of b - A u from level l to level l+1, with the
 * residual of the exactly solved cells taken as 0. */
cc_status cc_restrict_residual(cc_handle h, int level, const double* d_u, const double* d_b,
                               double* d_rc, cc_stream stream);
/* u += interpolation (Eq. 5.11) of e_c from level l+1 to level l. */
cc_status cc_prolong_add(cc_handle h, int level, const double* d_ec, double* d_u,
                         cc_stream stream);
/* One cycle of Alg. 2 (or its W form, as set up) on the finest level, u in
 * place, in the handle's cycle precision: FP64, or with CC_PREC_MIXED the
 * FP32 cycle of the mixed mode (u and b rounded to FP32 on entry, the
 * result widened to FP64; empty cells come back as the cycle left them). */
cc_status cc_cycle(cc_handle h, double* d_u, const double* d_b, cc_stream stream);

/*
 * cc_smooth_noalloc: the same block-smoother sweep as cc_smooth, for callers
 * that must not allocate device memory when they call it.  Such callers
 * include code running while a stream is being captured (cudaMalloc is not
 * allowed there), real-time loops that cannot afford an allocation's
 * latency or its implicit synchronisation, and hosts whose device memory is
 * owned by another allocator.  The paper has no counterpart: this only
 * changes where the sweep keeps its temporaries.
 *
 * The call allocates nothing and writes none of the handle's buffers.
 * The Jacobi output and the chunked block solve's temporaries (the
 * interface right-hand sides, the chunk interior solutions and the chunks'
 * contributions to the interface right-hand sides) live in one file-scope
 * device array of CC_NOALLOC_SCRATCH_DOUBLES doubles (8 MiB) in the
 * library.  Every GPU that loads the library's device code holds that array
 * until the process exits.  cc_setup looks up the array's device address
 * (cudaGetSymbolAddress) with the handle's device current and keeps it in
 * the handle (a clone shares it), so the call itself makes no runtime query
 * and may run inside a stream capture; a handle made after a device reset
 * holds the address in the new context.
 *
 * All calls share the one array, and it keeps the last call's contents.
 * Each call writes every entry it reads before reading it, so nothing needs
 * clearing between calls.  Calls that overlap on the GPU (on different
 * streams or different handles of one device) race on the array, so
 * serialise them.
 *
 *   level   0 .. n_levels - 2 (as for cc_smooth)
 *   d_u     N_l^2 FP64 values; input, and output of one sweep (empty cells 0)
 *   d_b     N_l^2 FP64 right-hand side
 * Errors: CC_ERR_ARG for a bad argument, a device other than the handle's,
 * or a level that needs more than CC_NOALLOC_SCRATCH_DOUBLES doubles
 * (N_l^2, plus for a chunked block its size, its interface count and its
 * contribution count; cc_last_error_string() gives the numbers).
 * CC_ERR_CUDA if the address lookup or a launch fails.  The call cannot
 * report a bounded wait that expires inside its kernels (a shared-memory
 * copy that never completes, which the library does not expect): such a
 * kernel gives up after about 0.1 s and leaves its rows of d_u unwritten.
 */
#define CC_NOALLOC_SCRATCH_DOUBLES (1 << 20)
cc_status cc_smooth_noalloc(cc_handle h, int level, double* d_u, const double* d_b,
                            cc_stream stream);

/*
 * cc_level_tables: copy level l's discretisation to host memory for
 * inspection.  Any pointer may be NULL.
 *   h_kind[N_l^2]     0 empty, 1 SFV, 2 PLG
 *   h_lattice[15*m]   the poised lattice (row-major cell indices) of each
 *                     PLG cell, PLG cells in row-major order (m = n_plg)
 *   h_beta[16*m]      beta_1..beta_15 and beta_b (0 for regular PLG cells)
 *   *n_plg            m
 */
cc_status cc_level_tables(cc_handle h, int level, uint8_t* h_kind, int* h_lattice,
                          double* h_beta, int* n_plg);

/*
 * cc_level_block: copy the cells of level l's exactly solved block (Eq. 5.8:
 * the PLG cells, and with b != 0 the SFV cells within 4 cells of a box
 * corner) in the solve order of Def. 5.1 to host memory (h_cells[m], may
 * be NULL); *m receives the count.
 */
cc_status cc_level_block(cc_handle h, int level, int* h_cells, int* m);

/* Kernels that cc_kernel_timing can time. */
enum { CC_TIME_OFF = 0, CC_TIME_FINE_SWEEP = 1, CC_TIME_BLOCK = 2, CC_TIME_FINE_BLOCK = 3 };

/*
 * cc_kernel_timing: with which = CC_TIME_FINE_SWEEP the library records CUDA
 * events around every launch of the finest-level Jacobi sweep kernel (Eq.
 * 5.7); with CC_TIME_BLOCK around every exact block solve (Eq. 5.8, any
 * level: its one launch, or its two chunked launches together); with
 * CC_TIME_FINE_BLOCK around the finest level's block solves only;
 * CC_TIME_OFF stops.  The events are recorded on the solve's stream, inside
 * its CUDA graph, so host launch gaps are not measured, but each interval
 * includes the launch latency of the kernels it brackets.
 * cc_kernel_timing_read returns the number of timed intervals, their total
 * milliseconds and, per interval, the average algorithmic bytes and the
 * average bytes the library's kernels actually move (either pointer may be
 * NULL), at the cycle's precision w:
 *   sweep        algorithmic = moved = 3 w per cell (u and b read, u written);
 *   block solve  algorithmic: the method's own price of the solve, the gather
 *                terms (column, coefficient, gathered value), b and the cell
 *                of every row, banded LU factors of 2 bw + 1 values per row
 *                (Def. 5.3, bw the block's bandwidth in curve order) and the
 *                writes; moved: the same gather and writes plus the dense
 *                inverse, or every chunk's two stages and the interface
 *                vectors.
 * Enabling resets the counters.  Errors: CC_ERR_ARG for an unknown kernel.
 */
cc_status cc_kernel_timing(cc_handle h, int which);
cc_status cc_kernel_timing_read(cc_handle h, int64_t* launches, double* total_ms,
                                double* bytes_per_launch, double* moved_bytes_per_launch);

#ifdef __cplusplus
}
#endif
#endif /* CCMG_H */
