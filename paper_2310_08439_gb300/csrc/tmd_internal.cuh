// Internal declarations of the GB300 TensorMD library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>
#include <cstdint>
#include <cstdio>
#include <string>

#include "tmd.h"

namespace tmd {

constexpr int NMOM = 20;        // moment components d, ranks 0..3 (Eq. T_dm)
constexpr int WARP = 32;
constexpr int MAX_LAYERS = TMD_MAX_HIDDEN + 1;

// Device status bits recorded by kernels, returned by synchronising calls.
enum : int32_t {
    DEV_ERR_OUTSIDE_BOX = 1,
    DEV_ERR_BAD_TYPE = 2,
    DEV_ERR_DEGREE = 4,
    DEV_ERR_SHIFT = 8,
    DEV_ERR_CELL = 16,
    DEV_ERR_TIMEOUT = 32,   // a bounded wait of a tensor-core kernel gave up
};

// Model as seen by kernels (passed by value).
struct DevModel {
    int S, K, L, act, Dd, nlayers, precision;
    float rc, rc2, inv_rc, sp_b;
    float rc2h, rc2l;                   // rc*rc as hi + lo (cutoff decision)
    int dims[MAX_LAYERS + 1];           // Dd, widths..., 1
    const float4 *radial;               // [S*S*K] (mu_hi, mu_lo, eta*log2(e), 2*eta)
    const float *wf[TMD_MAX_SPECIES];   // forward: per layer W^T [in][out], then b [out]
    const float *wb[TMD_MAX_SPECIES];   // backward: per layer W [out][in]
    const uint16_t *hf[TMD_MAX_SPECIES]; // BF16 forward copy (same layout as wf, no bias)
    const uint16_t *hb[TMD_MAX_SPECIES]; // BF16 backward copy (same layout as wb)
    int off_f[MAX_LAYERS];              // offset of layer l in wf[s] / hf[s]
    int off_b[MAX_LAYERS];              // offset of layer l in wb[s] / hb[s]
    // tile shapes (host-side launch choices; 0 = built-in default)
    int tile_rows;                      // atoms per FP32 network tile: 32 or 64 (streamed weights), 128 (resident)
    int pair_bps;                       // blocks per SM of the persistent pair-kernel grid
    // tabulated radial basis (nullptr = direct evaluation): per species pair
    // p = t_i S + t_j, rtab_n grid intervals [g, g + 1) / rtab_scale, each
    // holding per k the four cubic coefficients (c0, c1, c2, c3) of H in
    // t = r rtab_scale - g, the cutoff function folded in
    const float *rtab;
    float rtab_scale;                   // grid points per Angstrom (a power of two)
    int rtab_n;
    // BF16 weights in the tcgen05 operand layout (nullptr: not built): per
    // species, product p (forward layers, then the backward chain) at uoff[p]
    // elements, as [N pass][64-wide K chunk][N/8][8 core matrices][8 x 8]
    const uint16_t *ub[TMD_MAX_SPECIES];
    int uoff[2 * MAX_LAYERS];
};

// persistent grid of the pair kernels for n atoms
constexpr int PAIR_WARPS = 4;   // warps (atoms in flight) per block of the pair kernels
int pair_blocks(const DevModel &dm, int64_t n);
// shared memory of the FP32 network kernel with tr-atom tiles
size_t mlp_smem_tr_public(const DevModel &dm, int tr);
// tile_rows tr (32 / 64: streamed weights; 128: resident weights) can run this network
bool mlp_rows_ok(const DevModel &dm, int tr);
size_t mlp_bf16_smem_bytes(const DevModel &dm);
// tcgen05 form of the BF16 network (mlp_umma.cu)
bool mlp_umma_supported(const DevModel &dm);
tmd_status mlp_umma_launch(const DevModel &dm, const int32_t *perm, const int32_t *types, int64_t n, const float *G,
                           float *dG, float *e_atom, double *part_e, int *ntile_out, cudaStream_t s);
// network kernel of the BF16 form: 0 = tcgen05 when the shapes allow it, else
// mma.sync; 1 = tcgen05 only; 2 = mma.sync only
int network_kernel();
// force pass of the FP32 path: TMD_FORCE_AUTO / _SIMT / _TENSOR (api.cu)
int force_kernel();

// One system of a batch (a single evaluation is a batch of one): box, cell
// grid, first global cell, list radius and the FP32 screening band.
struct SysParams {
    double L[3];        // box lengths
    double ic[3];       // cells per unit length (nc / L)
    double r2;          // list radius squared (FP64, as the definition)
    float Lh[3], Ll[3]; // box as FP32 hi + lo (neighbour table build)
    float Gh[3], Gl[3]; // box on the 2^-10 grid split (pair kernels, grid_split)
    float r2lo, r2hi;   // FP32 band outside which the FP32 screen decides
    int nc[3], R[3], pbc[3];
    int cell_off;       // first global cell of this system
};

// v = hi + lo with hi = v rounded to a multiple of 2^-10 (exact in FP32 for
// |v| < 2^13) and lo = v - hi rounded to FP32 (|lo| <= 2^-11): differences of
// hi parts are exact in FP32, which keeps the pair geometry accurate without
// error-free transformations (pair_geom).
__host__ __device__ inline void grid_split(double v, float &hi, float &lo) {
    const double h = rint(v * 1024.0) * (1.0 / 1024.0);
    hi = (float)h;
    lo = (float)(v - h);
}
// largest |s| L, position or box length the grid split keeps exact
constexpr double GRID_LIMIT = 8192.0;

// Neighbour table as seen by kernels.
struct DevNlist {
    const int64_t *beg = nullptr;   // [n] first entry of atom a
    const int64_t *end = nullptr;   // [n] one past its last entry
    const int32_t *nbr = nullptr;   // [nnz]
    const char4 *shift = nullptr;   // [nnz] (sx, sy, sz, species of j)
    const int32_t *perm = nullptr;  // [n] atoms grouped by species, index order within a species
    const float4 *ph = nullptr;     // [n] positions, FP32 high part
    const float4 *pl = nullptr;     // [n] positions, FP32 low part (x = hi + lo)
    const SysParams *sp = nullptr;  // per-system boxes (batched), or nullptr
    const int32_t *sys_of = nullptr; // [atoms] system of each atom (batched), or nullptr
    double box[3] = {0, 0, 0};
    float Lh[3] = {0, 0, 0}, Ll[3] = {0, 0, 0};  // box on the 2^-10 grid split (single system)
    int64_t n = 0;                  // atoms in perm
    // in-cutoff pairs of atom a, compacted at [beg[a], beg[a] + npair[a]):
    // (Dx, Dy, Dz, j | b << 28) and r^2 as hi + lo; written by k_screen
    // when non-null, read by the descriptor and force passes
    float4 *pq = nullptr;
    float2 *pq2 = nullptr;
    int32_t *npair = nullptr;
};

}  // namespace tmd

struct tmd_model {
    tmd::DevModel dm;
    void *dev_block = nullptr;  // one allocation holding radial + all weights
    size_t dev_bytes = 0;
    int precision = TMD_PREC_FP32;
    float *dev_rtab = nullptr;  // tabulated radial basis (tmd_model_set_radial_table)
    void *dev_umma = nullptr;   // BF16 weights in the tcgen05 operand layout
    std::vector<double> mu, eta; // radial parameters [S][S][K] (host copy, for tables)
    double rc_exact = 0.0;
};

struct tmd_nlist {
    // geometry of the last build
    int64_t n = 0;
    double box[3] = {0, 0, 0};
    int32_t pbc[3] = {0, 0, 0};
    double r_list = 0;
    int nc[3] = {1, 1, 1};
    int R[3] = {1, 1, 1};
    int64_t ncell = 0;
    int64_t nnz = 0;
    int64_t n_active = 0;   // atoms binned and listed by the last build
    int built = 0;
    int32_t type_count[TMD_MAX_SPECIES] = {};

    // device arrays (capacities in elements)
    int32_t *cell_of = nullptr;      int64_t cap_atoms = 0;
    int32_t *cell_atoms = nullptr;   int64_t cap_cell_atoms = 0;
    float4 *cell_pos = nullptr;      int64_t cap_cell_pos = 0;
    int32_t *perm = nullptr;         int64_t cap_perm = 0;
    int64_t *beg = nullptr;          int64_t cap_beg = 0;          // [n] segment of atom i
    int64_t *end = nullptr;          int64_t cap_end = 0;          // [n]
    unsigned long long *counter = nullptr; int64_t cap_counter = 0;
    int32_t *cell_start = nullptr;   int64_t cap_cells = 0;
    int32_t *cell_fill = nullptr;    int64_t cap_cell_fill = 0;
    int32_t *nbr = nullptr;          int64_t cap_nnz = 0;
    char4 *shift = nullptr;          int64_t cap_shift = 0;
    int32_t *status = nullptr;       int64_t cap_status = 0;       // [1] device status bits
    int32_t *type_block = nullptr;   int64_t cap_type_blocks = 0;  // [blocks][8]: species counts, padded
    int32_t *type_start = nullptr;   int64_t cap_type_start = 0;   // [MAX_SPECIES + 1]
    tmd::SysParams *sp = nullptr;    int64_t cap_sp = 0;           // per-system parameters (device)
    int32_t *cell_sys = nullptr;     int64_t cap_cell_sys = 0;     // [ncell] system of each cell (batched)
    int32_t *todo = nullptr;         int64_t cap_todo = 0;         // atoms left to the per-atom pass
    unsigned long long *todo_count = nullptr; int64_t cap_todo_count = 0;
    int64_t *scan_tmp = nullptr;     int64_t cap_scan = 0;
    int64_t *h_pinned = nullptr;     // host pinned scratch (16 int64)

    // compute workspace
    float *G = nullptr;       int64_t cap_G = 0;    // [n][Dd]
    float *dG = nullptr;      int64_t cap_dG = 0;   // [n][Dd]
    float *P = nullptr;       int64_t cap_P = 0;    // [n][S][K][20]
    unsigned long long *Fq = nullptr; int64_t cap_Fq = 0; // [n][3] forces, 2^-32 fixed point
    float4 *ph = nullptr;     int64_t cap_ph = 0;   // [n] positions hi
    float4 *pl = nullptr;     int64_t cap_pl = 0;   // [n] positions lo
    double *part = nullptr;   int64_t cap_part = 0; // block partial sums
    float4 *pq = nullptr;     int64_t cap_pq = 0;   // [nnz] in-cutoff pair cache (geometry)
    float2 *pq2 = nullptr;    int64_t cap_pq2 = 0;  // [nnz] r^2 hi / lo
    int32_t *npair = nullptr; int64_t cap_npair = 0; // [n] in-cutoff pairs per atom
    int32_t *perm_own = nullptr; int64_t cap_perm_own = 0; // [n_owned] evaluation order of owned centres
    int32_t *own_count = nullptr; int64_t cap_own_count = 0; // [MAX_SPECIES] owned atoms per species

    // staging for the host-buffer entry point
    double *io_pos = nullptr;   int64_t cap_io_pos = 0;
    int32_t *io_types = nullptr; int64_t cap_io_types = 0;
    float *io_forces = nullptr; int64_t cap_io_forces = 0;
    double *io_red = nullptr;   int64_t cap_io_red = 0;   // energy + virial
};

namespace tmd {

// A captured CUDA graph of one fixed launch sequence, keyed by everything the
// sequence's launches depend on (buffer addresses, sizes, scalars).  The first
// call with a new key runs eagerly (it sizes the workspaces); the second
// captures and instantiates; later calls replay.
struct GraphCache {
    std::vector<uintptr_t> key, pending;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
    ~GraphCache() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

}  // namespace tmd

struct tmd_system {
    int64_t n = 0;
    double box[3];
    int32_t pbc[3];
    double skin = 0;
    double *pos = nullptr, *vel = nullptr, *pos_ref = nullptr, *inv_mass = nullptr, *mass = nullptr;
    int32_t *types = nullptr;
    float *forces = nullptr;
    double *red = nullptr;       // [32] device reduction outputs (E, W, KE, max disp)
    double *part = nullptr;      int64_t cap_part = 0;
    double *h_red = nullptr;     // host pinned mirror of red
    tmd_nlist nl;
    int64_t step = 0, rebuilds = 0;
    int need_rebuild = 1, have_forces = 0;
    tmd::GraphCache g_step;      // force evaluation + second half kick
    // runs of steps as one launch sequence (tmd_step): state at the start of
    // the run (for an exact rerun), skin-check flag of each step, host mirror
    double *snap_pos = nullptr, *snap_vel = nullptr;
    float *snap_forces = nullptr;
    int32_t *run_flags = nullptr;
    int64_t *h_run = nullptr;    // pinned: flags, entry counter, status
    tmd::GraphCache g_run;
    int64_t runs = 0, reruns = 0;
    int near_skin = 0;           // an atom moved more than 0.7 skin/2 since the last build
};

namespace tmd {

// Counts every kernel launch and, while profiling is enabled, records a pair
// of events around it on the launching stream.
class ProfScope {
   public:
    ProfScope(const char *name, cudaStream_t s);
    ~ProfScope();

   private:
    cudaStream_t stream_;
    int kernel_;
    cudaEvent_t start_;
};

// profiling switch and launch counter (kernels replayed from a CUDA graph
// are added to the counter by the replaying code)
bool profiling_on();
void add_launches(int64_t k);

#define TMD_LAUNCH(name, stream, ...)                   \
    do {                                                \
        ::tmd::ProfScope _prof_scope((name), (stream)); \
        __VA_ARGS__;                                    \
    } while (0)

// Thread-local error detail.
void set_error(const char *fmt, ...);
tmd_status cuda_fail(cudaError_t e, const char *what);

#define TMD_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return ::tmd::cuda_fail(_e, #call);       \
    } while (0)

// Grow a device buffer to at least `need` elements (contents discarded).
template <typename T>
tmd_status grow(T **ptr, int64_t *cap, int64_t need) {
    if (need <= *cap && *ptr) return TMD_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    int64_t n = need < 1 ? 1 : need;
    n = n + n / 8 + 16;
    cudaError_t e = cudaMalloc((void **)ptr, sizeof(T) * (size_t)n);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        set_error("cudaMalloc of %lld bytes failed: %s", (long long)(sizeof(T) * n), cudaGetErrorString(e));
        return TMD_ERR_OOM;
    }
    *cap = n;
    return TMD_OK;
}

void nlist_free(tmd_nlist *nl);

// Launchers (stream-ordered, no synchronisation unless stated).
// Per-system grid for a list radius (host); returns CAPACITY if the radius
// needs image shifts beyond +-15 boxes.
tmd_status make_sys_params(const double box[3], const int32_t pbc[3], double r_list, SysParams *sp, int64_t *ncell);
// Bin and list the atoms of the active systems (sys_of / active may be
// nullptr for a single system); synchronises once.  device_only: the same
// build with no host read and no allocation, for a stream capture; it needs
// a build with the same atoms and cells before, and the caller checks the
// entry counter against the capacity and the status word afterwards.
tmd_status build_tables(const double *pos, const int32_t *types, int64_t n, int n_sys, const SysParams *sp_host,
                        const int32_t *sys_of, const uint8_t *active, const int64_t *n_of_sys, int64_t ncell_total,
                        tmd_nlist *nl, cudaStream_t s, bool device_only = false);
// Evaluate the atoms listed by the last build_tables of nl (batched): per
// atom energies and virials, forces of the active atoms, per-system FP64
// reductions (energy, virial, m v v) for the active systems in act_list.
tmd_status run_compute_batch(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                             int64_t n_total, const int32_t *sys_of, float *forces, float *e_atom, float *w_atom,
                             const int32_t *act_list, int n_act, const int64_t *sys_off, const double *vel,
                             const double *mass, double *sys_out, cudaStream_t s);
void sys_reduce_launch(const int32_t *act, int n_act, const int64_t *off, const float *e_atom, const float *w_atom,
                       const double *vel, const double *mass, double *out, cudaStream_t s);
tmd_status build_neighbors(const double *pos, const int32_t *types, int64_t n, const double box[3],
                           const int32_t pbc[3], double r_list, tmd_nlist *nl, cudaStream_t s);
// descriptor (fwd) or force pass of one evaluation, one function per radial
// channel count K (pair_k<K>.cu); UNIMPLEMENTED for a species count without
// an instance
#define TMD_PAIR_LAUNCHER(name)                                                                            \
    tmd_status name(const DevModel &dm, const DevNlist &dn, const double *pos, const int32_t *types,       \
                    tmd_nlist *nl, double *part_w, int nblk, cudaStream_t s, bool fwd, float *w_atom)
TMD_PAIR_LAUNCHER(launch_pair_k8);
TMD_PAIR_LAUNCHER(launch_pair_k16);
TMD_PAIR_LAUNCHER(launch_pair_k32);
TMD_PAIR_LAUNCHER(launch_pair_k64);
TMD_PAIR_LAUNCHER(launch_pair_k128);
tmd_status reserve_compute(const DevModel &dm, tmd_nlist *nl, int64_t n_total, int64_t n_active);
// the in-cutoff pairs of the atoms of dn into its pair cache (screen.cu)
tmd_status launch_screen(const DevModel &dm, const DevNlist &dn, cudaStream_t s);
// BF16 weights in the tcgen05 operand layout from the FP64 weights (leaves
// dm.ub null when the widths have no BF16 form); status bits of the
// tensor-core kernels, read and cleared (synchronises)
tmd_status mlp_umma_build(tmd_model *m, const double *const *weights);
tmd_status umma_status(int32_t *bits);
tmd_status wait_probe(int32_t *gave_up);
extern int g_network_kernel;
// pos_split: the table's split positions (nl->ph, nl->pl) already hold pos
// (the MD step writes them in its drift); otherwise they are formed here
tmd_status run_compute(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                       int64_t n, const double box[3], double *energy, float *e_atom, float *forces,
                       double *virial, cudaStream_t s, bool pos_split = false);
tmd_status run_descriptors(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                           int64_t n, const double box[3], float *G, float *dEdG, cudaStream_t s);
// tmd_compute with atoms [n_owned, n) as ghosts: neighbours only, no energy
// term of their own (domain decomposition)
tmd_status run_compute_owned(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                             int64_t n, int64_t n_owned, const double box[3], double *energy, float *e_atom,
                             float *forces, double *virial, cudaStream_t s);
tmd_status run_compute_noalloc(const tmd_model *model, const int64_t *off, const int32_t *nbr, const int8_t *shift4,
                               int64_t nnz, const double *pos, const int32_t *types, int64_t n, const double box[3],
                               double *energy, float *e_atom, float *forces, double *virial, cudaStream_t s);

}  // namespace tmd
