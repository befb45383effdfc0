/*
 * tmd.h - C ABI of the GB300 (sm_103a) TensorMD energy / force / virial path.
 *
 * Method: TensorMD (arXiv 2310.08439), Sec. "The Tensor Formalism".  For every
 * atom a the library gathers the neighbours inside the cutoff, evaluates the
 * radial tensor H_abck = f_k(R) f_c(R), the moment tensor M_abcd (ranks 0..3,
 * Eq. T_dm), contracts P_abkd = sum_c H_abck M_abcd, forms the descriptor
 * G_abkm = sigma(T_dm P_abkd^2) (Eqs. tensor_formalism, sigma_function), runs
 * the per-species atomic-energy network E_a = NNP(G_a), and back-propagates
 * dE/dG through Eqs. dP_abkd, U_abck, F1_abcx, F2_abcx and the ScatterSum into
 * forces and the virial.  The neighbour table is built by cell binning with a
 * skin buffer (Sec. "Evaluation", binning with a 1 A buffer), and tmd_step
 * integrates with velocity-Verlet (1 fs steps in the paper).
 *
 * Conventions shared by every entry point
 *  - Units: A, eV, amu, fs.  Forces eV/A, virial eV, pressure eV/A^3.
 *  - Boxes are orthorhombic, box[3] = (Lx, Ly, Lz) > 0; pbc[x] != 0 marks a
 *    periodic axis.  Positions must lie in [0, L) on every axis (wrapped on
 *    periodic axes, inside the box on open ones).
 *  - Neighbour pairs: D_ij = x_j + s*L - x_i for an image shift s in Z^3;
 *    g_ij = dE/dD_ij; F_i += g_ij, F_j -= g_ij; W_ab = -sum_pairs D^a g^b.
 *  - "dev" pointers are CUDA device pointers on the current device; "host"
 *    pointers are ordinary host memory.  The caller owns every array it
 *    passes; the library owns its opaque handles and their workspaces.
 *  - Work is enqueued on the caller's stream and is asynchronous unless the
 *    description says the call synchronises.  A NULL stream is the legacy
 *    default stream.
 *  - Every call returns a tmd_status.  On error nothing is written to the
 *    caller's outputs beyond what is stated, and tmd_last_error() returns a
 *    human-readable reason (thread-local, valid until the next call).
 *  - Arguments are validated on the host before any launch.  Conditions only
 *    the device can see (an atom outside the box, a neighbour count above the
 *    list capacity) are recorded in a device status word and returned by the
 *    next call that synchronises (tmd_neighbors, tmd_nlist_*, tmd_step).
 *  - Host threads: calls from several threads must be serialised by the
 *    caller.  The library's one-time set-up (kernel shared-memory limits,
 *    occupancy queries) and its process-wide switches (tmd_set_graphs,
 *    tmd_set_network_kernel, tmd_set_force_kernel, profiling) are plain
 *    process state without locks; only the error string above is per thread.
 */
#ifndef TMD_H
#define TMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *tmd_stream_t; /* same handle as cudaStream_t */

typedef enum {
    TMD_OK = 0,
    TMD_ERR_INVALID_ARG = 1,   /* a host-side argument check failed            */
    TMD_ERR_CAPACITY = 2,      /* a size limit of the library was exceeded      */
    TMD_ERR_CUDA = 3,          /* a CUDA runtime call failed                    */
    TMD_ERR_OOM = 4,           /* device allocation failed                      */
    TMD_ERR_TIMEOUT = 5,       /* a bounded device wait gave up                 */
    TMD_ERR_UNIMPLEMENTED = 6  /* a configuration the library does not support  */
} tmd_status;

enum { TMD_ACT_TANH = 0, TMD_ACT_SQUAREPLUS = 1 };
enum { TMD_PREC_FP32 = 0, TMD_PREC_BF16 = 1 };
enum { TMD_NET_AUTO = 0, TMD_NET_TCGEN05 = 1, TMD_NET_MMA_SYNC = 2 };
/* force pass of the unbatched evaluation (tmd_set_force_kernel) */
enum { TMD_FORCE_AUTO = 0, TMD_FORCE_SIMT = 1, TMD_FORCE_TENSOR = 2 };

/* Limits of the library. */
#define TMD_MAX_SPECIES 5
#define TMD_MAX_HIDDEN 4
#define TMD_MAX_WIDTH 256
#define TMD_MAX_DEGREE 1024 /* neighbour entries per atom inside r_list */

/* Name of a status code (static string). */
const char *tmd_status_string(int status);
/* Detail of the last error raised on this thread ("" if none). */
const char *tmd_last_error(void);
/* Library version string. */
const char *tmd_version(void);

/* ------------------------------------------------------------------------ */
/* Potential model                                                          */
/* ------------------------------------------------------------------------ */
/*
 * Description of a TensorMD potential (all pointers host, read at create).
 *  n_species  S, 1..TMD_MAX_SPECIES.  Species ids are 0..S-1.
 *  n_radial   K radial channels; the library supports K in {8, 16, 32, 64,
 *             128} with at most 5, 5, 5, 2, 1 species respectively (the
 *             paper's pair-type index b runs over 1..5).
 *  rc         cutoff radius (A); pairs with R >= rc contribute nothing.
 *  mu, eta    [S][S][K] Gaussian centre and width of f_k(R) = exp(-eta (R-mu)^2)
 *             for (centre species, neighbour species, k).  f_c(R) =
 *             (cos(pi R / rc) + 1) / 2.  (H_abck definition; the paper leaves
 *             f_k open and names Gaussians as one choice.)
 *  n_hidden   L hidden layers, 1..TMD_MAX_HIDDEN; widths[L] each a multiple of
 *             4 and <= TMD_MAX_WIDTH.  Input width Dd = S*K*4, output 1.
 *  weights    [S] pointers; weights[s] holds, for l = 0..L, W_l [out][in]
 *             row-major then b_l [out] (FP64).  Descriptor column
 *             c = ((b*K) + k)*4 + m, b = neighbour species.
 *  activation TMD_ACT_TANH or TMD_ACT_SQUAREPLUS (b = squareplus_b); the
 *             output layer is linear.
 *  precision  TMD_PREC_FP32: every layer in FP32.  TMD_PREC_BF16: network
 *             layers on BF16 tensor cores with FP32 accumulation (input,
 *             activations and weights rounded to BF16; hidden widths must be
 *             multiples of 16, else TMD_ERR_UNIMPLEMENTED); radial basis,
 *             moments and contractions stay FP32 in both modes.
 */
typedef struct {
    int32_t n_species;
    int32_t n_radial;
    double rc;
    const double *mu;
    const double *eta;
    int32_t n_hidden;
    const int32_t *widths;
    const double *const *weights;
    int32_t activation;
    double squareplus_b;
    int32_t precision;
} tmd_model_desc;

typedef struct tmd_model tmd_model;   /* opaque; device copy of the weights */
typedef struct tmd_nlist tmd_nlist;   /* opaque; device neighbour table + workspace */
typedef struct tmd_system tmd_system; /* opaque; resident MD state */

/* Copy a model to the current device.  Errors: INVALID_ARG (bad sizes or a
 * non-finite weight), UNIMPLEMENTED (K or S outside the supported pairs, or a
 * network whose activations do not fit on chip), OOM, CUDA.
 * Synchronises the device once. */
tmd_status tmd_model_create(const tmd_model_desc *desc, tmd_model **out);
/* Free a model and its device memory (synchronises the device through
 * cudaFree).  NULL is accepted.  Always TMD_OK. */
tmd_status tmd_model_destroy(tmd_model *model);
/* Switch the network precision of an existing model (TMD_PREC_*). */
tmd_status tmd_model_set_precision(tmd_model *model, int32_t precision);

/* Tabulated radial basis (Sec. "The H_abck tensor and Batch Rational 1D
 * Interpolation": H_abck = f_k(R) f_c(R) and its derivative read from a
 * precomputed table instead of evaluating the Gaussians and the cutoff per
 * pair).  points_per_angstrom = 0 returns to direct evaluation (the default);
 * otherwise a power of two in [16, 1024].  Between grid points
 * R_g = g / points_per_angstrom the kernels interpolate H and H' with the
 * cubic Hermite polynomial through the exact H and H' at both ends (the paper
 * interpolates with rational functions; this reading uses the same table with
 * an O(h^4) error for H and O(h^3) for H', h = 1/ppa).  The table holds, for
 * every species pair and interval, the polynomial's four coefficients per k
 * (computed in FP64 on the host, stored FP32; H is zero from rc on):
 * [S][S][floor(rc*ppa)+2][K][4] floats on the device, owned by the model.
 * Errors: INVALID_ARG (ppa not 0 or a power of two in range), OOM/CUDA on
 * allocation or upload (the model is then back on direct evaluation).
 * Synchronises the device. */
tmd_status tmd_model_set_radial_table(tmd_model *model, int32_t points_per_angstrom);

/* Tabulated radial basis from the caller's own radial functions (the same
 * section: H_abck may come from any mapping of R, e.g. an embedding network,
 * once tabulated).  H, dH (host, FP64) [S][S][n_points][K]: H_k and dH_k/dR
 * for (centre species, neighbour species, k) at R_g = g / points_per_angstrom,
 * g = 0 .. n_points - 1; n_points >= ceil(rc * points_per_angstrom) (every
 * grid point below rc).  Values at R_g >= rc are ignored and taken as zero
 * (the cutoff is folded into the table: the caller's functions should go
 * smoothly to zero at rc).  Interpolation and storage as in
 * tmd_model_set_radial_table, which (or this call) replaces the previous
 * table; tmd_model_set_radial_table(model, 0) returns to the model's
 * Gaussians.  Errors: INVALID_ARG (ppa not a power of two in [16, 1024], NULL
 * arrays, too few points, a non-finite value), OOM/CUDA.  Synchronises. */
tmd_status tmd_model_set_radial_table_values(tmd_model *model, int32_t points_per_angstrom, int32_t n_points,
                                             const double *H, const double *dH);

/*
 * CUDA graphs (the paper has no counterpart: a launch-overhead measure of this
 * implementation).  The MD step loops (tmd_step, tmd_batch_step) and
 * tmd_batch_compute run their fixed evaluation sequence through a captured
 * CUDA graph: the first call with a given table layout, model and step size
 * runs eagerly, the second captures and instantiates, later calls replay.
 * Layout changes (a reallocated workspace, another set of active systems)
 * start over.  Graphs are never used on the legacy default stream (NULL),
 * while profiling is enabled, or after tmd_set_graphs(0) (process-wide;
 * default on).  tmd_graph_replays counts the replays so far.
 */
tmd_status tmd_set_graphs(int32_t on);

/* Network kernel of the BF16 form (process-wide; default TMD_NET_AUTO).  The
 * per-species network E_a = NNP(G_a) and its input gradient run either on the
 * fifth-generation tensor cores (tcgen05.mma into tensor memory, 128-atom
 * tiles, weights bulk-copied in 64-wide K chunks; needs every layer width a
 * multiple of 16, hidden widths <= 256, and the accumulators plus the stored
 * activation derivatives within 512 TMEM columns) or on mma.sync m16n8k16
 * (64-atom tiles).  AUTO takes tcgen05 when the shapes allow it;
 * TMD_NET_TCGEN05 makes other shapes fail with UNIMPLEMENTED, and so does
 * TMD_NET_MMA_SYNC for a network whose 64-atom mma.sync tile exceeds the
 * shared memory of an SM (reported by the evaluation call).  Both compute
 * BF16 products with FP32 accumulation (results differ in rounding order
 * only).  Errors: INVALID_ARG. */
tmd_status tmd_set_network_kernel(int32_t kind);

/* Force pass of the unbatched evaluation (process-wide; default
 * TMD_FORCE_AUTO = TMD_FORCE_SIMT).  The per-pair sums V_d = sum_k P'_kd H_k
 * and W_d = sum_k P'_kd H'_k (Eqs. U_abck, F1_abcx, F2_abcx) run either as
 * FP32 FMAs, one pair per lane (SIMT), or per atom as one matrix product
 * [H; H'] P' on the tensor cores (TENSOR: mma.sync on TF32 operands, each
 * operand split into two TF32 parts and three products accumulated in FP32,
 * which keeps FP32 accuracy).  TENSOR needs one species, K <= 32, the direct
 * radial basis and a table with the pair cache; other models then fail with
 * UNIMPLEMENTED.  Batched evaluations always use the SIMT pass.  Errors:
 * INVALID_ARG. */
tmd_status tmd_set_force_kernel(int32_t kind);

/* Status bits recorded by device kernels that have no neighbour table to
 * report through (today: a bounded wait of the tcgen05 network kernel that
 * gave up), read and cleared.  Returns TMD_ERR_TIMEOUT when such a wait ran
 * out since the last call (the results of the calls in between are invalid),
 * else TMD_OK; *bits receives the raw bits.  Synchronises the device. */
tmd_status tmd_device_status(int32_t *bits);

/* Self-test of the bounded waits of the tensor-core kernels: one warp
 * allocates tensor memory and waits, with the library's bounded wait, on an
 * mbarrier that nothing signals.  The wait gives up after about 0.2 s,
 * records the timeout (the next tmd_device_status returns TMD_ERR_TIMEOUT),
 * and the kernel frees its tensor memory and returns, leaving the context
 * usable.  *gave_up (host) = 1 when the wait gave up as designed.  Errors:
 * INVALID_ARG, CUDA.  Synchronises the device. */
tmd_status tmd_selftest_bounded_wait(int32_t *gave_up);
int64_t tmd_graph_replays(void);

/*
 * Tile shapes of this implementation's kernels (the paper has no counterpart:
 * they are launch choices of the GPU path).  32 and 64 give the same results
 * up to the order of FP64 partial sums; 128 runs the network's FP32 sums in
 * another order (results agree to FP32 rounding).
 *  tile_rows           atoms per tile of the FP32 network kernel: 32 or 64
 *                      (weights streamed through shared memory), 128
 *                      (weights resident in shared memory; networks whose
 *                      descriptor length and hidden widths are all 64, one or
 *                      two hidden layers; other networks fall back to the
 *                      built-in choice), 0 = built-in choice (128 where it
 *                      applies, else 32);
 *  pair_blocks_per_sm  blocks per SM of the persistent descriptor / force
 *                      grids (0 = built-in 16);
 *  ms                  output of the tuners: measured milliseconds of one
 *                      evaluation with these shapes (ignored on input).
 */
typedef struct {
    int32_t tile_rows;
    int32_t pair_blocks_per_sm;
    float ms;
} tmd_tuning;

/* Set / read a model's tile shapes.  set rejects tile_rows other than 0, 32,
 * 64, 128 and pair_blocks_per_sm outside [0, 64] (TMD_ERR_INVALID_ARG). */
tmd_status tmd_model_set_tuning(tmd_model *model, const tmd_tuning *tuning);
tmd_status tmd_model_get_tuning(const tmd_model *model, tmd_tuning *tuning);

/*
 * Autotuner: times tmd_compute on the caller's own system (dev pos [n][3],
 * dev types [n], built table nl) for every candidate tile shape (tile_rows
 * 32 / 64 where the shared memory allows it, 128 where the network allows
 * it, pair_blocks_per_sm 4, 8, 16,
 * 32), with CUDA events on the stream, keeps the fastest in the model and
 * writes it to *best (host).  Results computed while tuning are discarded.
 * Synchronises the stream.  Errors: as tmd_compute.
 */
tmd_status tmd_autotune(tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types, int64_t n,
                        const double box[3], tmd_tuning *best, tmd_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Neighbour table (R_abc of Sec. "The Tensor Formalism"; cell binning with */
/* a skin buffer, Sec. "Evaluation")                                        */
/* ------------------------------------------------------------------------ */
/* An empty table; device memory is taken by the first tmd_neighbors call
 * and grown as needed.  Errors: INVALID_ARG (out NULL), OOM.  destroy frees
 * it (NULL accepted; always TMD_OK). */
tmd_status tmd_nlist_create(tmd_nlist **out);
tmd_status tmd_nlist_destroy(tmd_nlist *nl);

/*
 * Build the neighbour table of n atoms: every (j, s) with
 * |x_j + s*L - x_i|^2 < r_list^2 and (j, s) != (i, 0), including periodic
 * self-images when a box side is shorter than 2*r_list.  The distance test
 * is decided in FP64 with the expression ((x_j + s*L) - x_i) per axis and
 * (dx*dx + dy*dy) + dz*dz, without fused multiply-add.  On the device each
 * atom's entries form one contiguous segment in a deterministic order (cell
 * stencil order, ascending atom id within a cell).
 *  pos    dev [n][3] FP64, in [0, L) per axis.
 *  types  dev [n] int32 species ids (< TMD_MAX_SPECIES).
 *  box    host [3]; pbc host [3].
 *  r_list list radius (cutoff + skin), > 0.
 * Allocates or grows nl's device arrays and synchronises the stream once (to
 * size the table).  Errors: INVALID_ARG (bad host argument, or an atom found
 * outside the box / an invalid species on the device), CAPACITY (an atom has
 * more than TMD_MAX_DEGREE entries or a shift beyond +-15 boxes), OOM, CUDA.
 */
tmd_status tmd_neighbors(const double *pos, const int32_t *types, int64_t n, const double box[3],
                         const int32_t pbc[3], double r_list, tmd_nlist *nl, tmd_stream_t stream);

/* Atom count and entry count of the last successful build (host outputs). */
tmd_status tmd_nlist_size(const tmd_nlist *nl, int64_t *n_atoms, int64_t *n_entries);

/*
 * Copy the table to host arrays in CSR form: off [n+1] int64 offsets, nbr
 * [nnz] int32 neighbour ids, shift [nnz][3] int8 image shifts, each atom's
 * entries ordered by (species of j, j, sx, sy, sz).  Any pointer may be NULL
 * to skip it.  Synchronises the device.
 */
tmd_status tmd_nlist_export(const tmd_nlist *nl, int64_t *off, int32_t *nbr, int8_t *shift);

/* ------------------------------------------------------------------------ */
/* Energy, forces, virial                                                   */
/* ------------------------------------------------------------------------ */
/*
 * E = sum_a E_a, E_a = NNP(G_a), F_ax = -dE/dx_ax, virial W (Sec. "The
 * Tensor Formalism": E_a, E, F_ax equations and the backward chain
 * Eqs. dP_abkd .. F2_abcx with ScatterSum).
 *  nl      a table built from the same positions' atoms and types with
 *          r_list >= model rc (a skin is allowed; entries beyond rc are
 *          skipped).  Its workspace is used and resized here.
 *  pos     dev [n][3] FP64; types dev [n] int32 (the ones given to
 *          tmd_neighbors); box host [3].
 *  energy  dev [1] FP64, sum of E_a accumulated in FP64.
 *  e_atom  dev [n] FP32 per-atom energies.
 *  forces  dev [n][3] FP32.
 *  virial  dev [9] FP64, row-major W_ab.
 * Any output may be NULL to skip it.  Asynchronous.  Errors: INVALID_ARG
 * (n differs from the table, r_list < rc), OOM, CUDA.
 */
tmd_status tmd_compute(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                       int64_t n, const double box[3], double *energy, float *e_atom, float *forces,
                       double *virial, tmd_stream_t stream);

/*
 * tmd_compute for one domain of a spatially decomposed system (the paper's
 * MPI decomposition, Sec. "Evaluation": each process evaluates the atoms of
 * its own domain with ghost copies of its neighbours' atoms).  Atoms
 * [0, n_owned) are owned centres; atoms [n_owned, n) are ghosts: copies of
 * other domains' atoms within the table radius of this domain, placed at the
 * image positions they have next to it.  Ghosts are neighbours of the centres
 * only: they have no energy term here (e_atom 0), and forces[ghost] holds the
 * ghost's share of the pair forces of this domain's centres, which the caller
 * adds to the forces of the atom the ghost copies (reverse exchange).
 * energy and virial sum over the owned centres, so the totals over domains
 * are those of the whole system.  Table and other arguments as tmd_compute
 * (the table is built over all n atoms).  Synchronises once (owned atoms per
 * species).  Errors: as tmd_compute; INVALID_ARG for n_owned outside [0, n].
 */
tmd_status tmd_compute_owned(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                             int64_t n, int64_t n_owned, const double box[3], double *energy, float *e_atom,
                             float *forces, double *virial, tmd_stream_t stream);

/*
 * Descriptor matrix G_abkm = sigma(T_dm (H_abck M_abcd)^2) (Eqs.
 * tensor_formalism, sigma_function), written to G dev [n][Dd] FP32, row a,
 * column ((b*K) + k)*4 + m.  When dEdG (dev [n][Dd] FP32) is non-NULL the
 * network is also run and its input gradient G'_abkm = dE_a/dG_abkm (the
 * quantity the backward chain starts from) is written there.  Same arguments
 * and errors as tmd_compute.  Asynchronous.
 */
tmd_status tmd_descriptors(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                           int64_t n, const double box[3], float *G, float *dEdG, tmd_stream_t stream);

/*
 * tmd_compute without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * while they run (codes that give all GPU memory to their own pool allocator
 * at start-up, or that must not allocate, or synchronise on an allocation,
 * inside their time-stepping loop).  The caller supplies the neighbour table
 * and every input and output; all scratch comes from one static device array
 * of 64 MiB (held by every GPU that loads the library until the process
 * exits), which bounds n: about 34,000 atoms for S=1, K=16 and about 18,000
 * for S=2, K=16 (beyond the bound the call returns TMD_ERR_CAPACITY before
 * touching the GPU).
 *  off      dev [n+1] int64 CSR offsets, off[0] = 0, off[n] = nnz.
 *  nbr      dev [nnz] int32 neighbour ids in [0, n).
 *  shift4   dev [nnz][4] int8 (sx, sy, sz, species of j), 4-byte aligned;
 *           the species byte must equal types[j]; |s| box < 4096 A on every
 *           axis; the table must hold every pair closer than rc (entries
 *           beyond rc are skipped).
 *  pos, types, box, energy, e_atom, forces, virial: as tmd_compute.
 * The first call on a device looks up the array's device address.  Each call
 * checks the table and the species on the device and synchronises the stream
 * once, before any force kernel runs, to read the result (TMD_ERR_INVALID_ARG
 * on a bad table).  It runs the SIMT force pass even when
 * tmd_set_force_kernel chose the tensor-core one (that pass reads a pair cache
 * this call does not keep).  Every call shares the one array and clears what
 * must start at zero; calls that overlap on the GPU (several streams or
 * threads at once) race on it and must be serialised by the caller.
 */
tmd_status tmd_compute_noalloc(const tmd_model *model, const int64_t *off, const int32_t *nbr, const int8_t *shift4,
                               int64_t nnz, const double *pos, const int32_t *types, int64_t n, const double box[3],
                               double *energy, float *e_atom, float *forces, double *virial, tmd_stream_t stream);

/*
 * One force evaluation from host buffers: copies pos [n][3] FP64 and types
 * [n] int32 from host memory (pinned memory gives asynchronous copies),
 * builds the table with r_list = rc, runs tmd_compute, and copies energy
 * (FP64 scalar), forces [n][3] FP32 and virial [9] FP64 back to host memory
 * (any output may be NULL).  Synchronises the stream before returning.
 */
tmd_status tmd_evaluate_host(const tmd_model *model, tmd_nlist *nl, const double *pos_host,
                             const int32_t *types_host, int64_t n, const double box[3],
                             const int32_t pbc[3], double *energy_host, float *forces_host,
                             double *virial_host, tmd_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Molecular dynamics (velocity-Verlet, NVE)                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    double e_pot;       /* potential energy, eV                        */
    double e_kin;       /* kinetic energy, eV                          */
    double temperature; /* K, from e_kin with 3n-3 degrees of freedom  */
    double virial[9];   /* eV                                          */
    double pressure[9]; /* (sum m v v + W) / V, eV/A^3                 */
    int64_t step;       /* steps taken since set_state                 */
    int64_t rebuilds;   /* neighbour rebuilds since set_state          */
} tmd_thermo;

/* Resident state of one system: n atoms in an orthorhombic box; the list
 * radius is rc + skin.  Allocates device memory.  Errors: INVALID_ARG, OOM. */
tmd_status tmd_system_create(int64_t n, const double box[3], const int32_t pbc[3], double skin,
                             tmd_system **out);
/* Free a system and its device and pinned host memory (NULL accepted;
 * always TMD_OK). */
tmd_status tmd_system_destroy(tmd_system *sys);

/*
 * Load positions [n][3] FP64 (A), velocities [n][3] FP64 (A/fs), types [n]
 * int32 and per-atom masses [n] FP64 (amu).  on_device != 0 means the
 * pointers are device pointers, else host.  vel and masses may be NULL
 * (zero velocities / unchanged masses).  Resets the step counter and forces a
 * neighbour rebuild.  Asynchronous on the stream.
 */
tmd_status tmd_system_set_state(tmd_system *sys, const double *pos, const double *vel,
                                const int32_t *types, const double *masses, int32_t on_device,
                                tmd_stream_t stream);
/* Copy positions / velocities [n][3] FP64 and forces [n][3] FP32 out (NULL
 * skips); on_device as above.  Synchronises the stream. */
tmd_status tmd_system_get_state(const tmd_system *sys, double *pos, double *vel, float *forces,
                                int32_t on_device, tmd_stream_t stream);
/* Host outputs (NULL skips): steps taken, table builds, runs of steps
 * completed as one launch sequence, and runs undone and stepped again one
 * step at a time (see tmd_step).  No GPU work. */
tmd_status tmd_system_counters(const tmd_system *sys, int64_t *steps, int64_t *rebuilds, int64_t *runs,
                               int64_t *reruns);

/*
 * Advance nsteps velocity-Verlet steps of dt_fs femtoseconds:
 *   v += dt/2 F/m; x += dt v; rebuild the table when rebuild_every > 0 and
 *   the step count is a multiple of it, or when any atom moved more than
 *   skin/2 since the last build (a rebuild first wraps the positions into the
 *   box); F = F(x); v += dt/2 F/m.  Between rebuilds positions are left
 *   unwrapped (they may lie up to skin/2 outside the box), because the
 *   table's image shifts refer to the positions at the last build.
 * (a = F/m * 1/103.6427 converts eV/(A amu) to A/fs^2.)  The first call after
 * set_state also computes the initial forces.  thermo (host, may be NULL)
 * receives the state after the last step.
 * With a skin and graphs on (tmd_set_graphs), steps run in runs decided on
 * the device: with rebuild_every > 0 from a cadence step to the step before
 * the next one (up to 16 steps), otherwise 16 steps at a time; a run is one
 * launch sequence (a captured graph on a non-default stream) whose cadence
 * rebuild runs on the device, and the host reads the skin flags of its steps
 * and the table's status once at the end.  A run in which an atom moved more
 * than skin/2 before a rebuild was due, or whose table overflowed, is undone
 * (its state was copied aside first) and stepped again one step at a time,
 * the host reading the skin flag after each step, so every trajectory is the
 * one that step-by-step path gives.  Steps outside runs synchronise once per
 * step.  Errors: as tmd_neighbors / tmd_compute.
 */
tmd_status tmd_step(const tmd_model *model, tmd_system *sys, double dt_fs, int32_t nsteps,
                    int32_t rebuild_every, tmd_thermo *thermo, tmd_stream_t stream);

/*
 * tmd_step from host buffers.  pos/vel [n][3] FP64 and forces_host [n][3]
 * FP32 are the caller's MD state in host memory (pinned memory gives
 * asynchronous copies).  The call uploads pos and vel, and the forces at pos
 * when forces_host is non-NULL (otherwise it recomputes them, with a
 * neighbour rebuild), runs nsteps steps as tmd_step does, and writes pos, vel
 * and forces back into the same host arrays.  The neighbour table follows
 * tmd_step's rules across calls (rebuild_every and the skin check); the skin
 * check compares the uploaded positions with those of the last build, so
 * positions the caller changed by more than skin/2 (a wrap included) force a
 * rebuild.  Synchronises the stream.
 */
tmd_status tmd_step_host(const tmd_model *model, tmd_system *sys, double *pos_host, double *vel_host,
                         float *forces_host, double dt_fs, int32_t nsteps, int32_t rebuild_every,
                         tmd_thermo *thermo, tmd_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batches: many independent systems resident at once (continuous batching) */
/* ------------------------------------------------------------------------ */
/*
 * A batch keeps n_systems independent periodic systems resident on the device
 * (concatenated atoms, one box per system).  Any subset of them is evaluated
 * or advanced by one set of launches: the cell list, neighbour table, pair
 * kernels and network run over the atoms of the listed systems only, each atom
 * using its own system's box, and energies / virials are reduced per system in
 * FP64.  Each system's energy, forces and virial are those of tmd_compute on
 * that system alone (the method is per system; Sec. "The Tensor Formalism").
 *
 * Neighbour tables stay resident between calls, one region of a shared entry
 * pool per system, built with r_list = rc + skin (tmd_batch_set_skin; skin 0,
 * the default, rebuilds the listed systems' tables on every evaluation).  A
 * system's table is rebuilt, alone or with the others due at the same step,
 * when it has none, on the cadence of rebuild_every steps, or when one of its
 * atoms moved more than skin / 2 since the build (the MD setting of Sec.
 * "Evaluation": binning with a 1 A buffer, rebuilt every 5 steps), as
 * tmd_step does for one system.  Positions are wrapped at each rebuild only.
 */
typedef struct tmd_batch tmd_batch;

/* n_atoms host [S] (>= 1 each), boxes host [S][3], pbc host [S][3].
 * Allocates the resident state.  Errors: INVALID_ARG, OOM. */
tmd_status tmd_batch_create(int32_t n_systems, const int64_t *n_atoms, const double *boxes, const int32_t *pbc,
                            tmd_batch **out);
/* Free a batch and its device and pinned host memory (NULL accepted;
 * always TMD_OK). */
tmd_status tmd_batch_destroy(tmd_batch *batch);
/* Load one system from host arrays: pos [n][3] FP64 (A), vel [n][3] FP64
 * (A/fs, NULL = zero), types [n] int32, masses [n] FP64 (amu).  Synchronises. */
tmd_status tmd_batch_set_system(tmd_batch *batch, int32_t sys, const double *pos, const double *vel,
                                const int32_t *types, const double *masses, tmd_stream_t stream);
/* Copy one system's positions / velocities (FP64 [n][3]) and forces (FP32
 * [n][3]) to host arrays (NULL skips).  Synchronises. */
tmd_status tmd_batch_get_system(const tmd_batch *batch, int32_t sys, double *pos, double *vel, float *forces,
                                tmd_stream_t stream);
/* Evaluate the listed systems (systems host [n_active], distinct ids):
 * energy host [n_active] FP64, virial host [n_active][9] FP64 (NULL skips);
 * forces stay resident (tmd_batch_get_system).  Synchronises once. */
tmd_status tmd_batch_compute(const tmd_model *model, tmd_batch *batch, const int32_t *systems, int32_t n_active,
                             double *energy, double *virial, tmd_stream_t stream);
/* Advance the listed systems by nsteps velocity-Verlet steps of dt_fs (as
 * tmd_step, with the batch's table policy; the skin criterion reads one flag
 * per system back once per step); thermo host [n_active] (may be NULL)
 * receives each system's state after the last step (rebuilds = that system's
 * table builds since tmd_batch_set_system).  Systems evaluated for the first
 * time get their initial forces first. */
tmd_status tmd_batch_step(const tmd_model *model, tmd_batch *batch, const int32_t *systems, int32_t n_active,
                          double dt_fs, int32_t nsteps, tmd_thermo *thermo, tmd_stream_t stream);

/* Table policy (no counterpart in the paper beyond its 1 A buffer and
 * 5-step cadence): skin >= 0 A added to rc for the tables, rebuild_every >= 0
 * steps (0 = the skin criterion only).  A new skin invalidates every table.
 * Errors: INVALID_ARG. */
tmd_status tmd_batch_set_skin(tmd_batch *batch, double skin, int32_t rebuild_every);
/* Give back system sys's table region (its pool entries are reused by the
 * next system that needs one); the system keeps its state and builds a new
 * table when it is next listed.  For servers that admit systems by device
 * memory: an idle system releases its table so that another can be admitted.
 * Errors: INVALID_ARG. */
tmd_status tmd_batch_release(tmd_batch *batch, int32_t sys);
/* Host outputs (NULL skips): entries of system sys's region (0 = none), of
 * the whole pool (its device memory is 8 B per entry for the table plus 24 B
 * for the in-cutoff pair cache), and the system's table builds. */
tmd_status tmd_batch_table_info(const tmd_batch *batch, int32_t sys, int64_t *region_entries,
                                int64_t *pool_entries, int64_t *rebuilds);

/*
 * Autotuner for batched evaluations: builds the tables of the listed systems
 * once, then times the batched force evaluation for every candidate tile shape
 * (as tmd_autotune) and keeps the fastest in the model; *best (host) receives
 * it.  The systems' positions are wrapped (as tmd_batch_compute does) but not
 * moved.  Synchronises the stream.
 */
tmd_status tmd_batch_autotune(tmd_model *model, tmd_batch *batch, const int32_t *systems, int32_t n_active,
                              tmd_tuning *best, tmd_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Profiling (per-kernel CUDA-event timing, launch counting)                */
/* ------------------------------------------------------------------------ */
typedef struct {
    char name[32];      /* kernel name                                         */
    int64_t launches;   /* launches recorded since the last reset              */
    double total_ms;    /* summed device time between the events around them   */
} tmd_kernel_stat;

/* Enable (on != 0) or disable event recording around every kernel launch of
 * the library.  The events are recorded on the launching stream, so the
 * durations are device times of each launch. */
tmd_status tmd_profile_enable(int32_t on);
/* Collect the recorded launches: waits for their events, writes at most cap
 * entries (one per kernel name that ran) and their number to *count, and
 * clears the records when reset != 0.  Synchronises on the recorded events. */
tmd_status tmd_profile_read(tmd_kernel_stat *out, int32_t cap, int32_t *count, int32_t reset);
/* Total number of kernel launches issued by the library in this process. */
int64_t tmd_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* TMD_H */
