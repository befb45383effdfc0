// TensorMD energy / force / virial evaluation for sm_103a: the network
// kernels and the host side of one evaluation.
//
// The paper's tensor diagram (Sec. "The Tensor Formalism") is evaluated as:
//   k_desc   setup, H, M, P = sum_c H M, G = sigma(T P^2)   (pair_kernels.cuh)
//   k_mlp    E_a = NNP(G_a) and G' = dE_a/dG_a    -- the E_a / NNP equations
//            (k_mlp_bf16: the same chain on BF16 tensor cores)
//   k_force  P', the pair gradients, ScatterSum, virial      (pair_kernels.cuh)
//   k_reduce FP64 energy and virial totals, k_forces_out int64 -> [n][3] FP32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "tmd_internal.cuh"
#include "net_common.cuh"

namespace tmd {

namespace {

constexpr int PW = PAIR_WARPS;  // warps per block in the pair kernels
constexpr int MT = 32;          // smallest network tile (sizes the per-tile energy partials)
constexpr int MLP_THREADS = 256;
constexpr double FQ_INV = 1.0 / 4294967296.0;   // forces accumulate in units of 2^-32 eV/A

// dst[perm[p]] = src[p] for rows of `width` floats (a multiple of 4): the
// per-atom view of a workspace kept in perm order
__global__ void k_rows_to_atoms(const float *__restrict__ src, const int32_t *__restrict__ perm, int64_t n, int width,
                                float *__restrict__ dst) {
    const int w4 = width >> 2;
    const int64_t total = n * w4;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / w4;
        const int c = (int)(t - p * w4);
        reinterpret_cast<float4 *>(dst + (size_t)perm[p] * width)[c] =
            reinterpret_cast<const float4 *>(src + (size_t)p * width)[c];
    }
}

// positions -> hi/lo FP32 pairs on the 2^-10 grid (grid_split; once per evaluation)
__global__ void k_split_pos(const double *__restrict__ pos, int64_t n, float4 *__restrict__ ph,
                            float4 *__restrict__ pl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h[3], l[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) grid_split(pos[3 * i + x], h[x], l[x]);
    ph[i] = make_float4(h[0], h[1], h[2], 0.f);
    pl[i] = make_float4(l[0], l[1], l[2], 0.f);
}

// ---------------------------------------------------------------------------
// network: E_a = NNP(G_a), G' = dE_a/dG_a (FP32 SIMT)
//
// A block of MLP_THREADS threads takes a tile of TR atoms in perm order (so a
// tile holds one species except at species boundaries).  Activations stay in
// shared memory transposed, [unit][atom] with row stride TR + 4, so a thread
// reads the 4 atoms of its row block for one unit with one vector load.  The
// weights are streamed through two shared-memory buffers in chunks of
// MLP_KC input rows by at most NP output columns: while the block multiplies
// with one chunk, cp.async brings in the next chunk of the tile's fixed
// sequence of products (forward layers, then the backward chain).  Every
// thread accumulates one 4 x 4 block of outputs per pass, summing each group
// of 16 products separately before adding it to the running total: the
// rounding error grows with 16 + Kin / 16 instead of Kin, which halves the
// error of G' for the 192-128-128 networks.  For one species the input
// activations are dead after the first product, so the second hidden layer
// takes their place (a smaller block, one more block per SM).
// ---------------------------------------------------------------------------
// streamed weight rows per chunk (32) and output columns per pass (64 for
// 64-atom tiles, 128 for 32-atom tiles): one 4 x 4 output block per thread
// and pass in both shapes
constexpr int MLP_KC = 32;
template <int TR>
__host__ __device__ constexpr int mlp_np() { return TR == 32 ? 128 : 64; }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// The products of one species, in order: step l < L is hidden layer l forward
// (A = a_l, B = W_l [in][out]); step L + t is the backward product for layer
// L - 1 - t (B = W^T [out][in]); the last one (layer 0) yields G'.
struct MlpStep {
    const float *W;
    int Kin, N;
};
__device__ __forceinline__ MlpStep mlp_step(const DevModel &m, int s, int step) {
    const int L = m.L;
    if (step < L) return {m.wf[s] + m.off_f[step], m.dims[step], m.dims[step + 1]};
    const int l = 2 * L - 1 - step;
    return {m.wb[s] + m.off_b[l], m.dims[l + 1], m.dims[l]};
}

// Issue the copy of chunk (n0, k0) of product st into buf (all threads).
template <int NP>
__device__ __forceinline__ void mlp_issue(const MlpStep &st, int n0, int k0, float *buf) {
    const int np = min(NP, st.N - n0), ncb = np >> 2, kc = min(MLP_KC, st.Kin - k0);
    if (np == st.N) {   // one contiguous block of W
        const float *src = st.W + (size_t)k0 * st.N;
        for (int idx = threadIdx.x; idx < kc * ncb; idx += MLP_THREADS) cp_async16(buf + 4 * idx, src + 4 * idx);
    } else {
        for (int idx = threadIdx.x; idx < kc * ncb; idx += MLP_THREADS) {
            const int kr = idx / ncb, c4 = idx - kr * ncb;
            cp_async16(buf + kr * np + 4 * c4, st.W + (size_t)(k0 + kr) * st.N + n0 + 4 * c4);
        }
    }
}

// Position in the weight stream: product st (sequence index step of species
// s), pass n0, chunk k0; buffer parity par.
struct MlpStream {
    int s, s_hi, step, n0, k0, par;
};

// Advance to the chunk after (n0, k0) of the current product (possibly the
// first chunk of the next product or species) and issue it; always commits a
// group so that wait_group 1 leaves exactly the current chunk pending.
template <int NP>
__device__ __forceinline__ void mlp_prefetch_next(const DevModel &m, const MlpStream &cur, const MlpStep &st,
                                                  float *wbuf) {
    int s = cur.s, step = cur.step, n0 = cur.n0, k0 = cur.k0 + MLP_KC;
    if (k0 >= st.Kin) {
        k0 = 0;
        n0 += NP;
        if (n0 >= st.N) {
            n0 = 0;
            if (++step == 2 * m.L) { step = 0; ++s; }
        }
    }
    if (s <= cur.s_hi) {
        const MlpStep nx = (step == cur.step && s == cur.s) ? st : mlp_step(m, s, step);
        mlp_issue<NP>(nx, n0, k0, wbuf + (cur.par ^ 1) * (MLP_KC * NP));
    }
    cp_async_commit();
}

// Activation buffers act[0..L] from base on (row stride ldt); returns the
// floats they take.  The input G (act[0]) is read by the first product only,
// so for a one-species model (one pass over the products per tile) act[2],
// written by the second product, shares its place.
__host__ __device__ inline size_t mlp_act_layout(const DevModel &m, int ldt, float *base, float **act) {
    const bool alias = m.S == 1 && m.L >= 2;
    size_t off = 0;
    for (int l = 0; l <= m.L; ++l) {
        if (alias && l == 2) {
            if (act) act[2] = act[0];
            continue;
        }
        if (act) act[l] = base + off;
        const int rows = (alias && l == 0 && m.dims[2] > m.dims[0]) ? m.dims[2] : m.dims[l];
        off += (size_t)rows * ldt;
    }
    return off;
}

// floats from the first activation buffer to act[l] in the layout above
__device__ __forceinline__ int mlp_act_offset(const DevModel &m, int ldt, int l) {
    const bool alias = m.S == 1 && m.L >= 2;
    if (alias && l == 2) l = 0;
    int off = 0;
    for (int q = 0; q < l; ++q) {
        if (alias && q == 2) continue;
        const int rows = (alias && q == 0 && m.dims[2] > m.dims[0]) ? m.dims[2] : m.dims[q];
        off += rows * ldt;
    }
    return off;
}

// One product of the stream.
// EPI 1: C^T[col][row] = act(acc + bias[col])           (hidden layer forward)
// EPI 2: C^T[col][row] = acc * act'(C^T[col][row])      (hidden layer backward, in place)
// EPI 3: gout[atom][col] = acc for rows of species s    (input gradient G')
template <int TR, int EPI>
__device__ __forceinline__ void mlp_gemm(const DevModel &m, MlpStream &ws, const float *At,
                                         const float *__restrict__ bias, float *Ct, float *wbuf,
                                         float *__restrict__ gout, const int *s_atom, const int *s_type) {
    constexpr int LDT = TR + 4;
    constexpr int NRB = TR / 4;    // row blocks
    constexpr int NP = mlp_np<TR>();
    static_assert(NRB * (NP / 4) == MLP_THREADS, "one 4 x 4 output block per thread and pass");
    const int tid = threadIdx.x;
    const MlpStep st = mlp_step(m, ws.s, ws.step);
    const int N = st.N;
    // row block fastest across the threads: conflict-free transposed loads and stores
    const int cb = tid / NRB, rb = tid - cb * NRB;
    for (int n0 = 0; n0 < N; n0 += NP) {
        const int np = min(NP, N - n0);
        const bool active = cb < (np >> 2);
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int o = 0; o < 4; ++o) acc[i][o] = 0.f;
        for (int k0 = 0; k0 < st.Kin; k0 += MLP_KC) {
            const int kc = min(MLP_KC, st.Kin - k0);
            ws.n0 = n0;
            ws.k0 = k0;
            mlp_prefetch_next<NP>(m, ws, st, wbuf);
            cp_async_wait1();
            __syncthreads();   // this chunk has landed for every thread; At is complete
            if (active && TR == 32) {
                // the same sums on packed FP32x2 multiply-adds (each half
                // rounds as fmaf): atom pairs (0, 1) and (2, 3) of the row
                // block against a duplicated weight
                const float *a = At + (size_t)k0 * LDT + rb * 4;
                const float *b = wbuf + ws.par * (MLP_KC * NP) + cb * 4;
                for (int kg = 0; kg < kc; kg += 16) {
                    float2 pp2[2][4];
#pragma unroll
                    for (int j = 0; j < 2; ++j)
#pragma unroll
                        for (int o = 0; o < 4; ++o) pp2[j][o] = make_float2(0.f, 0.f);
                    const int ke = min(kg + 16, kc);
                    auto step2 = [&](int k) {
                        const float4 av = *reinterpret_cast<const float4 *>(a + k * LDT);
                        const float4 bv = *reinterpret_cast<const float4 *>(b + k * np);
                        const float2 a01 = make_float2(av.x, av.y), a23 = make_float2(av.z, av.w);
                        const float bo[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                        for (int o = 0; o < 4; ++o) {
                            const float2 w2 = make_float2(bo[o], bo[o]);
                            pp2[0][o] = __ffma2_rn(a01, w2, pp2[0][o]);
                            pp2[1][o] = __ffma2_rn(a23, w2, pp2[1][o]);
                        }
                    };
                    if (ke - kg == 16) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) step2(kg + k);
                    } else {
                        for (int k = kg; k < ke; ++k) step2(k);
                    }
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        acc[0][o] += pp2[0][o].x;
                        acc[1][o] += pp2[0][o].y;
                        acc[2][o] += pp2[1][o].x;
                        acc[3][o] += pp2[1][o].y;
                    }
                }
            } else if (active) {
                // 64-atom tiles run four blocks per SM at 64 registers, where
                // the packed form's register pairs would cost a block
                const float *a = At + (size_t)k0 * LDT + rb * 4;
                const float *b = wbuf + ws.par * (MLP_KC * NP) + cb * 4;
                // groups of 16 products summed separately, then added to acc
                // (two-level summation; the same grouping for every tile
                // shape, so the result does not depend on it)
                for (int kg = 0; kg < kc; kg += 16) {
                    float pp[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int o = 0; o < 4; ++o) pp[i][o] = 0.f;
                    const int ke = min(kg + 16, kc);
                    auto step = [&](int k) {
                        const float4 av = *reinterpret_cast<const float4 *>(a + k * LDT);
                        const float4 bv = *reinterpret_cast<const float4 *>(b + k * np);
                        const float ai[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            pp[i][0] = fmaf(ai[i], bv.x, pp[i][0]);
                            pp[i][1] = fmaf(ai[i], bv.y, pp[i][1]);
                            pp[i][2] = fmaf(ai[i], bv.z, pp[i][2]);
                            pp[i][3] = fmaf(ai[i], bv.w, pp[i][3]);
                        }
                    };
                    if (ke - kg == 16) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) step(kg + k);
                    } else {
                        for (int k = kg; k < ke; ++k) step(k);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int o = 0; o < 4; ++o) acc[i][o] += pp[i][o];
                }
            }
            __syncthreads();   // every thread is done with this buffer
            ws.par ^= 1;
        }
        if (!active) continue;
        const int col = n0 + cb * 4;
        if (EPI == 3) {   // gout = the tile's first G' row (rows by perm position)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = rb * 4 + i;
                if (s_type[row] == ws.s)
                    *reinterpret_cast<float4 *>(gout + (size_t)row * N + col) =
                        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            }
        } else {
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                float *c = Ct + (size_t)(col + o) * LDT + rb * 4;
                float4 v;
                if (EPI == 1) {
                    const float bo = __ldg(bias + col + o);
                    v.x = act_f(m.act, acc[0][o] + bo, m.sp_b);
                    v.y = act_f(m.act, acc[1][o] + bo, m.sp_b);
                    v.z = act_f(m.act, acc[2][o] + bo, m.sp_b);
                    v.w = act_f(m.act, acc[3][o] + bo, m.sp_b);
                } else {
                    const float4 a = *reinterpret_cast<const float4 *>(c);
                    v.x = acc[0][o] * act_da(m.act, a.x, m.sp_b);
                    v.y = acc[1][o] * act_da(m.act, a.y, m.sp_b);
                    v.z = acc[2][o] * act_da(m.act, a.z, m.sp_b);
                    v.w = acc[3][o] * act_da(m.act, a.w, m.sp_b);
                }
                *reinterpret_cast<float4 *>(c) = v;
            }
        }
    }
    if (++ws.step == 2 * m.L) { ws.step = 0; ++ws.s; }
}

template <int TR>
__global__ void __launch_bounds__(MLP_THREADS, TR == 64 ? 4 : 2) k_mlp(DevModel m, const int32_t *__restrict__ perm,
                                                        const int32_t *__restrict__ types, int64_t n,
                                                        const float *__restrict__ G, float *__restrict__ dG,
                                                        float *__restrict__ e_atom, double *__restrict__ part_e) {
    constexpr int LDT = TR + 4;     // row stride of the transposed activations
    extern __shared__ __align__(16) float sm[];
    __shared__ int s_atom[TR], s_type[TR];
    __shared__ float s_e[TR];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * TR;
    const int L = m.L, Dd = m.Dd;
    // shared layout: two weight buffers, then act[l] = [dims[l]][LDT] for
    // l = 0..L, with act[2] over act[0] for a one-species model
    float *wbuf = sm;
    constexpr int NP = mlp_np<TR>();
    float *const abase = sm + 2 * MLP_KC * NP;
    // act[l]: computed where it is used (a pointer array indexed by the
    // runtime layer would live in local memory)
    auto act = [&](int l) -> float * { return abase + mlp_act_offset(m, LDT, l); };
    if (tid < TR) {
        const int64_t p = p0 + tid;
        const int a = p < n ? perm[p] : -1;
        s_atom[tid] = a;
        s_type[tid] = a >= 0 ? types[a] : -1;
        s_e[tid] = 0.f;
    }
    __syncthreads();
    int s_lo = TMD_MAX_SPECIES, s_hi = -1;
    for (int r = 0; r < TR; ++r)
        if (s_type[r] >= 0) { s_lo = min(s_lo, s_type[r]); s_hi = max(s_hi, s_type[r]); }
    MlpStream ws{s_lo, s_hi, 0, 0, 0, 0};
    if (s_lo <= s_hi) mlp_issue<NP>(mlp_step(m, s_lo, 0), 0, 0, wbuf);   // first chunk, under the G loads
    cp_async_commit();
    // G rows -> act[0] transposed (lane per atom row: conflict-free stores)
    float *const a0 = act(0);
    for (int r = lane; r < TR; r += 32) {
        const int a = s_atom[r];
        for (int c4 = warp; c4 < (Dd >> 2); c4 += MLP_THREADS / 32) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (a >= 0) v = __ldg(reinterpret_cast<const float4 *>(G + (size_t)(p0 + r) * Dd + 4 * c4));
            a0[(4 * c4) * LDT + r] = v.x;
            a0[(4 * c4 + 1) * LDT + r] = v.y;
            a0[(4 * c4 + 2) * LDT + r] = v.z;
            a0[(4 * c4 + 3) * LDT + r] = v.w;
        }
    }
    for (int s = s_lo; s <= s_hi; ++s) {
        const float *wf = m.wf[s], *wb = m.wb[s];
        for (int l = 0; l < L; ++l)
            mlp_gemm<TR, 1>(m, ws, act(l), wf + m.off_f[l] + m.dims[l] * m.dims[l + 1], act(l + 1), wbuf, nullptr,
                            s_atom, s_type);
        __syncthreads();
        // output layer (linear): E_r = b + w . a_L, then dz_L = w * act'(a_L) in place
        const int wl = m.dims[L];
        float *aL = act(L);
        const float *wout = wb + m.off_b[L];
        if (tid < TR) {
            float v0 = 0.f, v1 = 0.f;
            int c = 0;
            for (; c + 2 <= wl; c += 2) {
                v0 = fmaf(aL[c * LDT + tid], __ldg(wout + c), v0);
                v1 = fmaf(aL[(c + 1) * LDT + tid], __ldg(wout + c + 1), v1);
            }
            if (c < wl) v0 = fmaf(aL[c * LDT + tid], __ldg(wout + c), v0);
            if (s_type[tid] == s) {
                const float e = (v0 + v1) + __ldg(wf + m.off_f[L] + wl);
                s_e[tid] = e;
                if (e_atom) e_atom[s_atom[tid]] = e;
            }
        }
        __syncthreads();
        for (int c = warp; c < wl; c += MLP_THREADS / 32) {
            const float w = __ldg(wout + c);
            for (int r = lane; r < TR; r += 32) aL[c * LDT + r] = w * act_da(m.act, aL[c * LDT + r], m.sp_b);
        }
        // dz_l = (dz_{l+1} W_l^T) * act'(a_l), in place over a_l; B[k = o][n = i] = W_l[i][o]
        for (int l = L - 1; l >= 1; --l)
            mlp_gemm<TR, 2>(m, ws, act(l + 1), nullptr, act(l), wbuf, nullptr, s_atom, s_type);
        // G' = dz_1 W_0^T
        mlp_gemm<TR, 3>(m, ws, act(1), nullptr, nullptr, wbuf, dG + (size_t)p0 * Dd, s_atom, s_type);
    }
    asm volatile("cp.async.wait_all;\n" ::);
    __syncthreads();
    // tile energy in FP64, fixed order
    if (tid < 32) {
        double t = 0.0;
        for (int r = lane; r < TR; r += 32) t += (double)s_e[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) part_e[blockIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// network, FP32 SIMT with resident weights (E_a = NNP(G_a) and G' = dE_a/dG_a,
// Sec. "The Tensor Formalism"): networks whose descriptor length and hidden
// widths are all 64, with one or two hidden layers.
//
// A persistent block of 256 threads keeps one species' weight matrices in
// shared memory and walks a contiguous range of 128-atom tiles (perm order,
// so the species changes at most S - 1 times per block).  Every product of
// the chain (forward layers, then the input-gradient chain) is
// [128 x 64] x [64 x 64]: each thread owns an 8 x 4 block of the result
// (atoms 4 rb .. 4 rb + 3 and 64 + 4 rb .. 64 + 4 rb + 3, columns 4 cb ..
// 4 cb + 3) and runs 32 multiply-adds (16 packed FP32x2 instructions) per
// two float4 activation loads and one float4 weight load.  Each weight matrix is stored once in 4 x 4
// blocks: the forward products read rows of a block, the backward products
// (which multiply by W^T) read its columns from the same copy after loading
// the whole block.  The rows inside a block are XOR-swizzled so that the
// four column groups of a warp read distinct banks in both directions.  The
// output layer (E_a and dz_L) is formed in the epilogue of the last forward
// product.
//
// Two activation buffers X and Y alternate their roles from tile to tile.
// A tile starts with its G rows already in X (row-major, copied by cp.async
// while the previous tile ran its last product); they are transposed into Y,
// and the chain runs Y -> X (a_1) -> Y (dz_2) -> X (dz_1 over a_1) -> G'
// (one hidden layer: Y -> X (dz_1) -> G').  The last product reads only X,
// so the next tile's G rows are copied into Y meanwhile, and Y becomes the
// next tile's X.
// ---------------------------------------------------------------------------
constexpr int RW_TR = 128;              // atoms per tile
constexpr int RW_THREADS = 256;         // 8 warps, an 8 x 4 result block per thread
constexpr int RW_N = 64;                // descriptor length and every hidden width
constexpr int RW_LDT = RW_TR + 4;       // row stride of the transposed activations
constexpr int RW_LDG = RW_N + 4;        // row stride of staged G rows (conflict-free float4 reads)
constexpr int RW_MAXL = 2;              // hidden layers
constexpr int RW_WF = RW_N * RW_N;      // floats per weight matrix
constexpr int RW_BUF = (RW_N * RW_LDT > RW_TR * RW_LDG) ? RW_N * RW_LDT : RW_TR * RW_LDG;
constexpr int RW_CG = 4;                // column groups: energy partials of a row come from 4 warp pairs

// dynamic shared memory: weights, two activation buffers, biases, output
// weights and bias, the energy partials of the column groups
constexpr size_t RW_SMEM_FLOATS =
    (size_t)RW_MAXL * RW_WF + 2 * (size_t)RW_BUF + RW_MAXL * RW_N + RW_N + 4 + RW_CG * RW_TR;

// place of element (k, o) of a 64 x 64 matrix in the blocked, swizzled layout
__device__ __forceinline__ int rw_widx(int k, int o) {
    const int kb = k >> 2, ob = o >> 2, f = (kb ^ (ob >> 1)) & 3;
    return ((kb * 16 + ob) << 4) + (((k & 3) ^ f) << 2) + (o & 3);
}

__device__ __forceinline__ float rw_comp(const float4 v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// acc[i][c] = sum_k At[k][atom i] B[k][4 cb + c] over k = 0..63, where B = W
// (forward: W stored [in][out]) or B = W^T (backward).  The multiply-adds run
// on packed FP32x2 (fma.rn.f32x2, each half rounded as fmaf): atom pairs
// (i, i + 1) against a duplicated weight, so one instruction does two.
template <bool BWD>
__device__ __forceinline__ void rw_product(const float *At, const float *Wm, int rb, int cb, float (&acc)[8][4]) {
    float2 acc2[4][4];   // acc2[j][c] = (acc[2 j][c], acc[2 j + 1][c])
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2[j][c] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int g = 0; g < RW_N / 4; ++g) {
        // forward: block (g, cb), row k & 3 for k = 4 g .. 4 g + 3;
        // backward: block (cb, g), column k & 3
        const float *bk = Wm + (BWD ? 16 * (16 * cb + g) : 16 * (16 * g + cb));
        const int f = BWD ? ((cb ^ (g >> 1)) & 3) : ((g ^ (cb >> 1)) & 3);
        float4 w[4];   // logical rows 0..3 of the block
#pragma unroll
        for (int r = 0; r < 4; ++r) w[r] = *reinterpret_cast<const float4 *>(bk + 4 * (r ^ f));
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float *a = At + (4 * g + r) * RW_LDT + 4 * rb;
            const float4 a0 = *reinterpret_cast<const float4 *>(a);
            const float4 a1 = *reinterpret_cast<const float4 *>(a + 64);
            const float2 ap[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                                  make_float2(a1.z, a1.w)};
            float wv[4];
            if (!BWD) {
                wv[0] = w[r].x; wv[1] = w[r].y; wv[2] = w[r].z; wv[3] = w[r].w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) wv[q] = rw_comp(w[q], r);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float2 w2 = make_float2(wv[c], wv[c]);
#pragma unroll
                for (int j = 0; j < 4; ++j) acc2[j][c] = __ffma2_rn(ap[j], w2, acc2[j][c]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc[2 * j][c] = acc2[j][c].x;
            acc[2 * j + 1][c] = acc2[j][c].y;
        }
}

// the 8 atoms of a thread's result block as two float4 of a transposed row
__device__ __forceinline__ void rw_store_col(float *Ct, int col, int rb, const float (&v)[8]) {
    float *c = Ct + col * RW_LDT + 4 * rb;
    *reinterpret_cast<float4 *>(c) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4 *>(c + 64) = make_float4(v[4], v[5], v[6], v[7]);
}

// weights of species s into shared memory: W_l blocked (rw_widx), biases,
// output weights and bias
__device__ __forceinline__ void rw_load_species(const DevModel &m, int s, float *sW, float *sBias, float *sWout,
                                                float *sBout) {
    const int L = m.L;
    for (int l = 0; l < L; ++l) {
        const float *W = m.wf[s] + m.off_f[l];   // [64 in][64 out], then the bias [64]
        for (int idx = threadIdx.x; idx < RW_N * (RW_N / 4); idx += RW_THREADS) {
            const int k = idx >> 4, o = 4 * (idx & 15);
            *reinterpret_cast<float4 *>(sW + l * RW_WF + rw_widx(k, o)) =
                __ldg(reinterpret_cast<const float4 *>(W + k * RW_N + o));
        }
        if (threadIdx.x < RW_N) sBias[l * RW_N + threadIdx.x] = __ldg(W + RW_WF + threadIdx.x);
    }
    const float *wo = m.wf[s] + m.off_f[L];   // output layer: [64][1], then its bias
    if (threadIdx.x < RW_N) sWout[threadIdx.x] = __ldg(wo + threadIdx.x);
    if (threadIdx.x == 0) sBout[0] = __ldg(wo + RW_N);
}

// half h (threadIdx.x >> 7) of the G row at perm position p0 + (threadIdx.x
// & 127) (zeros beyond n) -> the staging buffer (row-major, stride RW_LDG),
// by cp.async; not waited for
__device__ __forceinline__ void rw_stage_g(const float *__restrict__ G, int64_t p0, int64_t n, float *X) {
    const int row = threadIdx.x & (RW_TR - 1), h = threadIdx.x >> 7;
    const int64_t p = p0 + row;
    const bool ok = p < n;
    const float *src = ok ? G + (size_t)p * RW_N + 32 * h : G;
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(X + row * RW_LDG + 32 * h);
    const int bytes = ok ? 16 : 0;   // 0: the 16 bytes are zero-filled
#pragma unroll
    for (int c4 = 0; c4 < 8; ++c4)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst + 16 * c4),
                     "l"(src + (ok ? 4 * c4 : 0)), "r"(bytes));
    cp_async_commit();
}

__global__ void __launch_bounds__(RW_THREADS, 2) k_mlp_res(DevModel m, const int32_t *__restrict__ perm,
                                                        const int32_t *__restrict__ types, int64_t n,
                                                        const float *__restrict__ G, float *__restrict__ dG,
                                                        float *__restrict__ e_atom, double *__restrict__ part_e) {
    extern __shared__ __align__(16) float sm[];
    float *sW = sm;                                  // L blocked 64 x 64 matrices
    float *buf0 = sW + RW_MAXL * RW_WF;              // the two activation buffers
    float *sBias = buf0 + 2 * RW_BUF;                // [L][64]
    float *sWout = sBias + RW_MAXL * RW_N;           // [64]
    float *sBout = sWout + RW_N;                     // [1] (+ 3 pad)
    float *sEp = sBout + 4;                          // [RW_CG][RW_TR]
    // per tile parity: atoms, species, energies and the warps' species
    // ranges (a tile's are written during the previous tile's last product)
    __shared__ int s_atom2[2][RW_TR], s_type2[2][RW_TR];
    __shared__ float s_e2[2][RW_TR];
    __shared__ int s_lohi2[2][RW_THREADS / 32][2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rb = (lane & 7) + 8 * (warp & 1), cb = (lane >> 3) + 4 * (warp >> 1);
    const int L = m.L, act = m.act;
    const float spb = m.sp_b;
    const int64_t ntile = (n + RW_TR - 1) / RW_TR;
    const int64_t t_beg = ntile * blockIdx.x / gridDim.x, t_end = ntile * (blockIdx.x + 1) / gridDim.x;
    int loaded = -1;   // species whose weights are in sW
    int xb = 0;        // buffer holding the tile's staged G rows
    float acc[8][4];
    // atoms and species of tile t at parity par (threads >= RW_TR only take
    // part in the warp reductions)
    auto publish = [&](int par, int a, int ty) {
        if (tid < RW_TR) {
            s_atom2[par][tid] = a;
            s_type2[par][tid] = ty;
            s_e2[par][tid] = 0.f;
        }
        const int lo = __reduce_min_sync(0xffffffffu, ty >= 0 ? ty : TMD_MAX_SPECIES);
        const int hi = __reduce_max_sync(0xffffffffu, ty);
        if (lane == 0) { s_lohi2[par][warp][0] = lo; s_lohi2[par][warp][1] = hi; }
    };
    if (t_beg < t_end) {
        rw_stage_g(G, t_beg * RW_TR, n, buf0);
        const int64_t p = t_beg * RW_TR + tid;
        const int a = (tid < RW_TR && p < n) ? perm[p] : -1;
        publish(0, a, a >= 0 ? types[a] : -1);
        __syncthreads();
    }
    for (int64_t tile = t_beg; tile < t_end; ++tile) {
        const int64_t p0 = tile * RW_TR;
        float *X = buf0 + xb * RW_BUF, *Y = buf0 + (xb ^ 1) * RW_BUF;
        const int *s_atom = s_atom2[xb], *s_type = s_type2[xb];
        float *s_e = s_e2[xb];
        const bool more = tile + 1 < t_end;
        int next_a = -1, next_ty = -1;   // the next tile's atom and species of this thread's row
        asm volatile("cp.async.wait_all;\n" ::);   // this thread's staged G row (read by it alone)
        int s_lo = TMD_MAX_SPECIES, s_hi = -1;
#pragma unroll
        for (int w = 0; w < RW_THREADS / 32; ++w) {
            s_lo = min(s_lo, s_lohi2[xb][w][0]);
            s_hi = max(s_hi, s_lohi2[xb][w][1]);
        }
        for (int s = s_lo; s <= s_hi; ++s) {
            if (s != s_lo) {   // a second species in this tile: its G rows again (X was overwritten)
                __syncthreads();
                rw_stage_g(G, p0, n, X);
                asm volatile("cp.async.wait_all;\n" ::);
                __syncthreads();
            }
            if (s != loaded) {
                rw_load_species(m, s, sW, sBias, sWout, sBout);
                loaded = s;
            }
            if (s == s_hi && more && tid < RW_TR) {   // read ahead: the next tile's atom (used before G')
                const int64_t p = p0 + RW_TR + tid;
                next_a = p < n ? perm[p] : -1;
            }
            {   // half of G row (tid & 127) (X, row-major) -> Y transposed (conflict-free both ways)
                const int row = tid & (RW_TR - 1), h = tid >> 7;
                const float *xr = X + row * RW_LDG + 32 * h;
#pragma unroll
                for (int c4 = 0; c4 < 8; ++c4) {
                    const float4 v = *reinterpret_cast<const float4 *>(xr + 4 * c4);
                    const int k = 32 * h + 4 * c4;
                    Y[k * RW_LDT + row] = v.x;
                    Y[(k + 1) * RW_LDT + row] = v.y;
                    Y[(k + 2) * RW_LDT + row] = v.z;
                    Y[(k + 3) * RW_LDT + row] = v.w;
                }
            }
            __syncthreads();
            // forward layers: G (Y) -> a_1 (X); the last one also forms E_a
            // and dz_L = w act'(a_L): L = 1 writes dz_1 into X, L = 2 writes
            // dz_2 into Y (G is dead)
            for (int l = 0; l < L; ++l) {
                const float *Ain = (l == 0) ? Y : X;
                float *Cout = (l == 0) ? X : Y;
                rw_product<false>(Ain, sW + l * RW_WF, rb, cb, acc);
                const float4 bv = *reinterpret_cast<const float4 *>(sBias + l * RW_N + 4 * cb);
                const float bias[4] = {bv.x, bv.y, bv.z, bv.w};
                if (l < L - 1) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float v[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) v[i] = act_f(act, acc[i][c] + bias[c], spb);
                        rw_store_col(Cout, 4 * cb + c, rb, v);
                    }
                    __syncthreads();
                } else {
                    const float4 wv = *reinterpret_cast<const float4 *>(sWout + 4 * cb);
                    const float wout[4] = {wv.x, wv.y, wv.z, wv.w};
                    float ep[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) ep[i] = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float v[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float a = act_f(act, acc[i][c] + bias[c], spb);
                            ep[i] = fmaf(a, wout[c], ep[i]);
                            v[i] = wout[c] * act_da(act, a, spb);
                        }
                        rw_store_col(Cout, 4 * cb + c, rb, v);
                    }
                    // E partials over this thread's 4 columns -> the 4 column
                    // groups of the warp (lanes 8 apart) -> the 4 warp pairs
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        ep[i] += __shfl_xor_sync(0xffffffffu, ep[i], 8);
                        ep[i] += __shfl_xor_sync(0xffffffffu, ep[i], 16);
                    }
                    if ((lane >> 3) == 0) {
                        float *e = sEp + (warp >> 1) * RW_TR + 4 * rb;
                        *reinterpret_cast<float4 *>(e) = make_float4(ep[0], ep[1], ep[2], ep[3]);
                        *reinterpret_cast<float4 *>(e + 64) = make_float4(ep[4], ep[5], ep[6], ep[7]);
                    }
                    __syncthreads();
                    if (tid < RW_TR && s_type[tid] == s) {
                        const float e = ((sEp[tid] + sEp[RW_TR + tid]) + (sEp[2 * RW_TR + tid] + sEp[3 * RW_TR + tid])) +
                                        sBout[0];
                        s_e[tid] = e;
                        if (e_atom) e_atom[s_atom[tid]] = e;
                    }
                }
            }
            // L = 2: dz_1 = (dz_2 W_1^T) act'(a_1), written over a_1 (each
            // thread reads and writes only its own block)
            if (L == 2) {
                rw_product<true>(Y, sW + RW_WF, rb, cb, acc);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float *cp = X + (4 * cb + c) * RW_LDT + 4 * rb;
                    const float4 a0 = *reinterpret_cast<const float4 *>(cp);
                    const float4 a1 = *reinterpret_cast<const float4 *>(cp + 64);
                    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    float v[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = acc[i][c] * act_da(act, av[i], spb);
                    rw_store_col(X, 4 * cb + c, rb, v);
                }
                __syncthreads();
            }
            // Y is free from here on: the next tile's G rows go there while
            // the last product runs
            if (s == s_hi && more) {
                rw_stage_g(G, p0 + RW_TR, n, Y);
                if (next_a >= 0) next_ty = types[next_a];
            }
            // G' = dz_1 W_0^T -> dG rows of species s (perm position)
            rw_product<true>(X, sW, rb, cb, acc);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int row = (i < 4) ? 4 * rb + i : 64 + 4 * rb + (i - 4);
                if (s_type[row] == s)
                    *reinterpret_cast<float4 *>(dG + (size_t)(p0 + row) * RW_N + 4 * cb) =
                        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            }
        }
        if (more) publish(xb ^ 1, next_a, next_ty);
        __syncthreads();   // every thread is done with X and s_e; the next tile's atoms are visible
        if (warp == 0) {   // tile energy in FP64, fixed order
            double t = 0.0;
            for (int r = lane; r < RW_TR; r += 32) t += (double)s_e[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) part_e[tile] = t;
        }
        xb ^= 1;
    }
    asm volatile("cp.async.wait_all;\n" ::);
}

// ---------------------------------------------------------------------------
// network on BF16 tensor cores (FP32 accumulation): the same forward / input-
// gradient chain as k_mlp for a 64-atom tile.  Eight warps: warp w owns rows
// 16 (w % 4) .. + 16 and one half of each weight chunk's output columns, and
// issues mma m16n8k16 with ldmatrix operands.  Activations and activation
// derivatives stay in shared memory as BF16; the weights stream through two
// shared buffers in chunks of BF_NC output rows (cp.async, one chunk ahead,
// across the whole product sequence).  The output layer (E_a) and dz_L are
// formed in the epilogue of the last forward product.
// ---------------------------------------------------------------------------
constexpr int BT = 64;            // atoms per BF16 tile
constexpr int BF_THREADS = 256;   // 8 warps: 4 row slabs x 2 column halves
constexpr int BF_NC = 64;         // output columns per streamed weight chunk (fewer for wide inputs)

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const uint16_t *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

// Product `step` of species s as Bt[n][k] (K contiguous per output column):
// forward layer l: Bt = W_l [out][in]; backward layer l: Bt = W_l^T [in][out].
struct BfStep {
    const uint16_t *Bt;
    int K, N;
};
__device__ __forceinline__ BfStep bf_step(const DevModel &m, int s, int step) {
    const int L = m.L;
    if (step < L) return {m.hb[s] + m.off_b[step], m.dims[step], m.dims[step + 1]};
    const int l = 2 * L - 1 - step;
    return {m.hf[s] + m.off_f[l], m.dims[l + 1], m.dims[l]};
}

// Bt rows [n0, n0 + min(bnc, N - n0)) into buf (row stride K + 8), one
// warp per row in 16-byte copies
__device__ __forceinline__ void bf_issue(const BfStep &st, int n0, int bnc, uint16_t *buf) {
    const int nc = min(bnc, st.N - n0), c8 = st.K >> 3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < nc; r += BF_THREADS / 32)
        for (int c = lane; c < c8; c += 32)
            cp_async16(buf + r * (st.K + 8) + 8 * c, st.Bt + (size_t)(n0 + r) * st.K + 8 * c);
}

__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, const uint16_t *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

struct BfStream {
    int s, s_hi, step, par;
};

__global__ void __launch_bounds__(BF_THREADS, 3) k_mlp_bf16(DevModel m, const int32_t *__restrict__ perm,
                                                         const int32_t *__restrict__ types, int64_t n,
                                                         const float *__restrict__ G, float *__restrict__ dG,
                                                         float *__restrict__ e_atom, double *__restrict__ part_e,
                                                         int bnc, int compact) {
    // bnc: output columns per streamed weight chunk (BF_NC, or 32 / 16 when
    // the input is wide enough that two BF_NC-column buffers would not fit).
    // compact != 0 (wide inputs, at least two hidden layers): the gradient
    // buffers reuse the G tile, which is dead after the first product, and
    // the G tile is loaded again for each further species of the tile.
    extern __shared__ __align__(16) uint16_t smh[];
    __shared__ int s_atom[BT], s_type[BT], s_range[2];
    __shared__ float s_e[BT], s_epart[2][BT];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int slab = warp & 3, half = warp >> 2;
    const int64_t p0 = (int64_t)blockIdx.x * BT;
    const int L = m.L, Dd = m.Dd;
    int maxw = 0, kmax = Dd;
    for (int l = 1; l <= L; ++l) {
        maxw = max(maxw, m.dims[l]);
        kmax = max(kmax, m.dims[l]);
    }
    // shared layout (BF16 elements): two weight buffers, act[0] = G tile,
    // act[l] / der[l] for hidden layers 1..L-1, two gradient buffers
    const int ldw_max = kmax + 8;
    uint16_t *wbuf = smh;
    uint16_t *act[MAX_LAYERS + 1], *der[MAX_LAYERS + 1];
    int ld[MAX_LAYERS + 1];
    uint16_t *ptr = smh + 2 * bnc * ldw_max;
    for (int l = 0; l < L; ++l) {
        ld[l] = m.dims[l] + 8;
        act[l] = ptr;
        ptr += BT * ld[l];
        der[l] = ptr;
        ptr += (l > 0) ? BT * ld[l] : 0;
    }
    const int ldz = maxw + 8;
    uint16_t *dzA = compact ? act[0] : ptr;
    uint16_t *dzB = dzA + BT * ldz;
    if (tid < BT) {
        const int64_t p = p0 + tid;
        const int a = p < n ? perm[p] : -1;
        s_atom[tid] = a;
        s_type[tid] = a >= 0 ? types[a] : -1;
        s_e[tid] = 0.f;
    }
    __syncthreads();
    if (warp == 0) {   // species present in the tile (perm groups atoms by species)
        int lo = TMD_MAX_SPECIES, hi = -1;
        for (int r = lane; r < BT; r += 32)
            if (s_type[r] >= 0) { lo = min(lo, s_type[r]); hi = max(hi, s_type[r]); }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) { s_range[0] = lo; s_range[1] = hi; }
    }
    __syncthreads();
    const int s_lo = s_range[0], s_hi = s_range[1];
    BfStream ws{s_lo, s_hi, 0, 0};
    if (s_lo <= s_hi) bf_issue(bf_step(m, s_lo, 0), 0, bnc, wbuf);   // first chunk, under the G loads
    cp_async_commit();
    // G rows -> act[0] as BF16 (warp per atom row)
    auto load_G = [&]() {
        for (int r = warp; r < BT; r += BF_THREADS / 32) {
            const int a = s_atom[r];
            for (int c2 = lane; c2 < (Dd >> 1); c2 += 32) {
                float2 v = make_float2(0.f, 0.f);
                if (a >= 0) v = __ldg(reinterpret_cast<const float2 *>(G + (size_t)(p0 + r) * Dd + 2 * c2));
                *reinterpret_cast<uint32_t *>(act[0] + r * ld[0] + 2 * c2) = pack_bf16(v.x, v.y);
            }
        }
    };
    load_G();
    for (int s = s_lo; s <= s_hi; ++s) {
        // every warp passed the barrier after the previous species' last chunk
        if (compact && s > s_lo) load_G();
        const float *wf = m.wf[s];
        const float *wout = m.wb[s] + m.off_b[L];
        float epart[2] = {0.f, 0.f};   // E partial sums of rows g and g + 8 (last forward product)
        uint16_t *cur = dzA, *nxt = dzB;
        for (int step = 0; step < 2 * L; ++step) {
            const BfStep st = bf_step(m, s, step);
            const bool fwd = step < L, last_fwd = step == L - 1, last = step == 2 * L - 1;
            const int l_out = fwd ? step + 1 : 2 * L - 1 - step;   // layer whose activation / gradient is formed
            const uint16_t *A = fwd ? act[step] : cur;
            const int lda = fwd ? ld[step] : ldz;
            const int ldw = st.K + 8;
            for (int n0 = 0; n0 < st.N; n0 += bnc) {
                // next chunk of the stream (same product, next product or next species)
                {
                    int s2 = s, step2 = step, n2 = n0 + bnc;
                    if (n2 >= st.N) {
                        n2 = 0;
                        if (++step2 == 2 * L) { step2 = 0; ++s2; }
                    }
                    if (s2 <= s_hi) bf_issue(bf_step(m, s2, step2), n2, bnc, wbuf + (ws.par ^ 1) * (bnc * ldw_max));
                    cp_async_commit();
                }
                cp_async_wait1();
                __syncthreads();   // this chunk has landed; A is complete
                const uint16_t *w = wbuf + ws.par * (bnc * ldw_max);
                const int nc = min(bnc, st.N - n0);
                const int hc = nc >> 1;                // columns of this warp's half
                const int nt = hc >> 3;                // n-tiles of 8 (1..4)
                float acc[4][4];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
                const uint16_t *pa = A + (slab * 16 + (lane & 15)) * lda + (lane >> 4) * 8;
                const uint16_t *pb = w + (half * hc + (lane & 7) + ((lane >> 4) << 3)) * ldw + ((lane >> 3) & 1) * 8;
                for (int k0 = 0; k0 < st.K; k0 += 16) {
                    uint32_t a0, a1, a2, a3;
                    ldsm_x4(a0, a1, a2, a3, pa + k0);
#pragma unroll
                    for (int j = 0; j < 4; j += 2) {
                        if (j + 1 < nt) {
                            uint32_t b0, b1, b2, b3;
                            ldsm_x4(b0, b1, b2, b3, pb + j * 8 * ldw + k0);
                            mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
                            mma_bf16(acc[j + 1], a0, a1, a2, a3, b2, b3);
                        } else if (j < nt) {   // a single n-tile (lanes 0-15 give the addresses)
                            uint32_t b0, b1;
                            ldsm_x2(b0, b1, pb + j * 8 * ldw + k0);
                            mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
                        }
                    }
                }
                // epilogue: element (row, col) of this lane is acc[j][2 h + e],
                // row = 16 slab + g + 8 h, col = n0 + half * hc + 8 j + 2 t + e
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j >= nt) continue;
                    const int col = n0 + half * hc + 8 * j + 2 * t;
                    if (fwd) {
                        const float b0 = __ldg(wf + m.off_f[step] + st.K * st.N + col);
                        const float b1 = __ldg(wf + m.off_f[step] + st.K * st.N + col + 1);
                        float w0 = 0.f, w1 = 0.f;
                        if (last_fwd) { w0 = __ldg(wout + col); w1 = __ldg(wout + col + 1); }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int row = slab * 16 + g + 8 * h;
                            float a0v, a1v, d0, d1;
                            act_fd_bf16(m.act, acc[j][2 * h] + b0, m.sp_b, a0v, d0);
                            act_fd_bf16(m.act, acc[j][2 * h + 1] + b1, m.sp_b, a1v, d1);
                            if (last_fwd) {   // E_r partial and dz_L = w_out * act'(a_L)
                                epart[h] = fmaf(w0, a0v, fmaf(w1, a1v, epart[h]));
                                *reinterpret_cast<uint32_t *>(dzA + row * ldz + col) = pack_bf16(w0 * d0, w1 * d1);
                            } else {
                                *reinterpret_cast<uint32_t *>(act[l_out] + row * ld[l_out] + col) = pack_bf16(a0v, a1v);
                                *reinterpret_cast<uint32_t *>(der[l_out] + row * ld[l_out] + col) = pack_bf16(d0, d1);
                            }
                        }
                    } else {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int row = slab * 16 + g + 8 * h;
                            if (!last) {   // dz_l = (dz_{l+1} W_l^T) * act'(a_l)
                                const float2 d = unpack_bf16(*reinterpret_cast<const uint32_t *>(der[l_out] + row * ld[l_out] + col));
                                *reinterpret_cast<uint32_t *>(nxt + row * ldz + col) =
                                    pack_bf16(acc[j][2 * h] * d.x, acc[j][2 * h + 1] * d.y);
                            } else if (s_type[row] == s) {   // G'
                                *reinterpret_cast<float2 *>(dG + (size_t)(p0 + row) * Dd + col) =
                                    make_float2(acc[j][2 * h], acc[j][2 * h + 1]);
                            }
                        }
                    }
                }
                __syncthreads();   // every warp is done with this weight buffer and with A
                ws.par ^= 1;
            }
            if (last_fwd) {
                // E_r = b + w . a_L: reduce the quad (the four lanes of a row), then the two halves
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    epart[h] += __shfl_xor_sync(0xffffffffu, epart[h], 1);
                    epart[h] += __shfl_xor_sync(0xffffffffu, epart[h], 2);
                    if (t == 0) s_epart[half][slab * 16 + g + 8 * h] = epart[h];
                }
                __syncthreads();
                if (tid < BT && s_type[tid] == s) {
                    const float e = (s_epart[0][tid] + s_epart[1][tid]) + __ldg(wf + m.off_f[L] + m.dims[L]);
                    s_e[tid] = e;
                    if (e_atom) e_atom[s_atom[tid]] = e;
                }
            }
            if (!fwd) { uint16_t *tmp = cur; cur = nxt; nxt = tmp; }
        }
    }
    asm volatile("cp.async.wait_all;\n" ::);
    __syncthreads();
    // tile energy in FP64, fixed order
    if (tid < 32) {
        double tsum = 0.0;
        for (int r = lane; r < BT; r += 32) tsum += (double)s_e[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
        if (lane == 0) part_e[blockIdx.x] = tsum;
    }
}

// FP64 totals of the block partials, fixed order (deterministic): RED_BLOCKS
// blocks each sum a fixed slice into RED_PART scratch doubles, then one warp
// adds those in block order.
constexpr int RED_BLOCKS = 64;
constexpr int RED_PART = RED_BLOCKS * 10;

__global__ void __launch_bounds__(256) k_reduce_part(const double *__restrict__ part_e, int ne,
                                                     const double *__restrict__ part_w, int nw,
                                                     double *__restrict__ red) {
    __shared__ double s[10][8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ce = (ne + RED_BLOCKS - 1) / RED_BLOCKS, cw = (nw + RED_BLOCKS - 1) / RED_BLOCKS;
    const int e0 = min(ne, (int)blockIdx.x * ce), e1 = min(ne, e0 + ce);
    const int w0 = min(nw, (int)blockIdx.x * cw), w1 = min(nw, w0 + cw);
    double v[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) v[t] = 0.0;
    for (int i = e0 + tid; i < e1; i += blockDim.x) v[0] += part_e[i];
    for (int i = w0 + tid; i < w1; i += blockDim.x)
#pragma unroll
        for (int t = 0; t < 9; ++t) v[1 + t] += part_w[(size_t)i * 9 + t];
#pragma unroll
    for (int t = 0; t < 10; ++t) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[t] += __shfl_xor_sync(0xffffffffu, v[t], o);
        if (lane == 0) s[t][warp] = v[t];
    }
    __syncthreads();
    if (tid < 10) {
        double acc = 0.0;
        for (int w = 0; w < 8; ++w) acc += s[tid][w];
        red[blockIdx.x * 10 + tid] = acc;
    }
}

__global__ void k_reduce(const double *__restrict__ red, double *__restrict__ energy, double *__restrict__ virial) {
    const int t = threadIdx.x;
    if (t >= 10) return;
    double acc = 0.0;
    for (int b = 0; b < RED_BLOCKS; ++b) acc += red[b * 10 + t];
    if (t == 0) { if (energy) *energy = acc; }
    else if (virial) virial[t - 1] = acc;
}

__global__ void k_forces_out(const long long *__restrict__ Fq, int64_t n, float *__restrict__ forces) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3 * n) forces[i] = (float)((double)Fq[i] * FQ_INV);
}

// forces of the atoms listed in perm (batched: only the active systems' atoms)
__global__ void k_forces_out_perm(const long long *__restrict__ Fq, const int32_t *__restrict__ perm, int64_t n,
                                  float *__restrict__ forces) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t a = perm[p];
    forces[3 * a] = (float)((double)Fq[3 * a] * FQ_INV);
    forces[3 * a + 1] = (float)((double)Fq[3 * a + 1] * FQ_INV);
    forces[3 * a + 2] = (float)((double)Fq[3 * a + 2] * FQ_INV);
}

// Per-system FP64 sums over each active system's atom range (one block per
// system, fixed order): out[b] = (E, W[9], sum m v_a v_b [xx yy zz xy xz yz]).
__global__ void k_sys_reduce(const int32_t *__restrict__ act, const int64_t *__restrict__ off,
                             const float *__restrict__ e_atom, const float *__restrict__ w_atom,
                             const double *__restrict__ vel, const double *__restrict__ mass, double *__restrict__ out) {
    __shared__ double s[16][8];
    const int sys = act[blockIdx.x];
    const int64_t beg = off[sys], end = off[sys + 1];
    double v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = 0.0;
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
        v[0] += (double)e_atom[i];
#pragma unroll
        for (int t = 0; t < 9; ++t) v[1 + t] += (double)w_atom[i * 9 + t];
        if (vel) {
            const double m = mass[i], x = vel[3 * i], y = vel[3 * i + 1], z = vel[3 * i + 2];
            v[10] += m * x * x; v[11] += m * y * y; v[12] += m * z * z;
            v[13] += m * x * y; v[14] += m * x * z; v[15] += m * y * z;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[t] += __shfl_xor_sync(0xffffffffu, v[t], o);
        if (lane == 0) s[t][warp] = v[t];
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        double acc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += s[threadIdx.x][w];
        out[(size_t)blockIdx.x * 16 + threadIdx.x] = acc;
    }
}

tmd_status dispatch_pair(const DevModel &dm, const DevNlist &dn, const double *pos, const int32_t *types,
                         tmd_nlist *nl, double *part_w, int nblk, cudaStream_t s, bool fwd, float *w_atom = nullptr) {
    switch (dm.K) {
    case 8: return launch_pair_k8(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    case 16: return launch_pair_k16(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    case 32: return launch_pair_k32(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    case 64: return launch_pair_k64(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    case 128: return launch_pair_k128(dm, dn, pos, types, nl, part_w, nblk, s, fwd, w_atom);
    default: break;
    }
    set_error("no kernel for K=%d S=%d", dm.K, dm.S);
    return TMD_ERR_UNIMPLEMENTED;
}

int sm_count() {
    static int count = 0;
    if (!count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
        if (count <= 0) count = 132;
    }
    return count;
}

}  // namespace

int pair_blocks(const DevModel &dm, int64_t n) {
    const int bps = dm.pair_bps > 0 ? dm.pair_bps : 16;
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + PW - 1) / PW, (int64_t)sm_count() * bps));
}

namespace {

}  // namespace

tmd_status run_compute_batch(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                             int64_t n_total, const int32_t *sys_of, float *forces, float *e_atom, float *w_atom,
                             const int32_t *act_list, int n_act, const int64_t *sys_off, const double *vel,
                             const double *mass, double *sys_out, cudaStream_t s);

static size_t mlp_bf16_smem_cfg(const DevModel &dm, int bnc, bool compact) {
    int maxw = 0, kmax = dm.Dd;
    for (int l = 1; l <= dm.L; ++l) {
        maxw = std::max(maxw, dm.dims[l]);
        kmax = std::max(kmax, dm.dims[l]);
    }
    size_t el = (size_t)2 * bnc * (kmax + 8);              // two weight buffers
    el += (size_t)BT * (dm.dims[0] + 8);                   // G tile
    for (int l = 1; l < dm.L; ++l) el += 2 * (size_t)BT * (dm.dims[l] + 8);   // act, act'
    if (!compact) el += 2 * (size_t)BT * (maxw + 8);       // gradient buffers
    return el * sizeof(uint16_t);
}

// launch shape of k_mlp_bf16: weight-chunk columns (BF_NC, 32 or 16) and
// whether the gradient buffers share the G tile, the first that fits an SM
struct BfCfg {
    int bnc;
    bool compact;
};
static BfCfg mlp_bf16_cfg(const DevModel &dm) {
    int maxw = 0;
    for (int l = 1; l <= dm.L; ++l) maxw = std::max(maxw, dm.dims[l]);
    const bool can_compact = dm.L >= 2 && dm.Dd + 8 >= 2 * (maxw + 8);
    for (int c = 0; c < (can_compact ? 2 : 1); ++c)
        for (int bnc = BF_NC; bnc >= 16; bnc >>= 1)
            if (mlp_bf16_smem_cfg(dm, bnc, c == 1) <= 227 * 1024) return {bnc, c == 1};
    return {16, can_compact};
}

size_t mlp_bf16_smem_bytes(const DevModel &dm) {
    const BfCfg c = mlp_bf16_cfg(dm);
    return mlp_bf16_smem_cfg(dm, c.bnc, c.compact);
}

// dynamic shared memory of k_mlp<TR>: transposed activations of every layer
// plus one staged weight chunk
static size_t mlp_smem_tr(const DevModel &dm, int tr) {
    size_t fl = mlp_act_layout(dm, tr + 4, nullptr, nullptr);
    fl += (size_t)2 * MLP_KC * (tr == 32 ? mlp_np<32>() : mlp_np<64>());   // two weight chunks
    return fl * sizeof(float);
}

// atoms per tile of the streamed-weight kernel: the tuning's 32 or 64, else
// 32 (its inner product runs on packed FP32x2 multiply-adds)
static int mlp_tr(const DevModel &dm) {
    if ((dm.tile_rows == 32 || dm.tile_rows == 64) && mlp_smem_tr(dm, dm.tile_rows) <= 227 * 1024) return dm.tile_rows;
    return 32;
}

size_t mlp_smem_bytes(const DevModel &dm) { return mlp_smem_tr(dm, mlp_tr(dm)); }

size_t mlp_smem_tr_public(const DevModel &dm, int tr) { return mlp_smem_tr(dm, tr); }

// the resident-weight FP32 network applies: descriptor length and hidden
// widths all 64, one or two hidden layers, 16-byte aligned weight rows
static bool mlp_res_ok(const DevModel &dm) {
    if (dm.precision != TMD_PREC_FP32 || dm.L < 1 || dm.L > RW_MAXL || dm.dims[dm.L + 1] != 1) return false;
    for (int l = 0; l <= dm.L; ++l)
        if (dm.dims[l] != RW_N || dm.off_f[l] % 4 != 0) return false;
    for (int s = 0; s < dm.S; ++s)
        if (reinterpret_cast<uintptr_t>(dm.wf[s]) % 16 != 0) return false;
    return true;
}

// tile_rows 0 (built-in choice) or 128 selects it where it applies
static bool mlp_use_res(const DevModel &dm) { return (dm.tile_rows == 0 || dm.tile_rows == RW_TR) && mlp_res_ok(dm); }

bool mlp_rows_ok(const DevModel &dm, int tr) {
    if (tr == RW_TR) return mlp_res_ok(dm);
    return (tr == 32 || tr == 64) && mlp_smem_tr(dm, tr) <= 227 * 1024;
}

static tmd_status validate(const tmd_model *model, tmd_nlist *nl, int64_t n, const double box[3]) {
    if (!model || !nl) {
        set_error("null model or neighbour table");
        return TMD_ERR_INVALID_ARG;
    }
    if (!nl->built || nl->n != n) {
        set_error("neighbour table was built for %lld atoms, compute called with %lld", (long long)nl->n,
                  (long long)n);
        return TMD_ERR_INVALID_ARG;
    }
    const DevModel &dm = model->dm;
    if (nl->r_list < (double)dm.rc * (1.0 - 1e-12)) {
        set_error("neighbour table radius %.6g is below the model cutoff %.6g", nl->r_list, (double)dm.rc);
        return TMD_ERR_INVALID_ARG;
    }
    for (int x = 0; x < 3; ++x)
        if (box[x] != nl->box[x]) {
            set_error("box differs from the one the neighbour table was built with");
            return TMD_ERR_INVALID_ARG;
        }
    for (int t = dm.S; t < TMD_MAX_SPECIES; ++t)
        if (nl->type_count[t] != 0) {
            set_error("species id %d present but the model has %d species", t, dm.S);
            return TMD_ERR_INVALID_ARG;
        }
    return TMD_OK;
}

// opt-in shared memory of the network kernel that runs: the FP32 k_mlp<TR>,
// or (bf16 = true) the mma.sync kernel of the BF16 form
static tmd_status set_mlp_smem(const DevModel &dm, bool bf16) {
    static size_t smem_set[2] = {0, 0}, smem_bf_set = 0;
    if (bf16) {
        const size_t sb = mlp_bf16_smem_bytes(dm);
        if (sb > 227 * 1024) {
            set_error("network too wide for the mma.sync BF16 kernel (%zu bytes of shared memory)", sb);
            return TMD_ERR_UNIMPLEMENTED;
        }
        if (sb > 48 * 1024 && sb > smem_bf_set) {
            TMD_CUDA(cudaFuncSetAttribute(k_mlp_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
            smem_bf_set = sb;
        }
        return TMD_OK;
    }
    if (mlp_use_res(dm)) return TMD_OK;   // k_mlp_res sets its own
    const int tr = mlp_tr(dm);
    const size_t smem = mlp_smem_bytes(dm);
    size_t &done = smem_set[tr == 64 ? 1 : 0];
    if (smem > 48 * 1024 && smem > done) {
        if (tr == 64)
            TMD_CUDA(cudaFuncSetAttribute(k_mlp<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        else
            TMD_CUDA(cudaFuncSetAttribute(k_mlp<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        done = smem;
    }
    return TMD_OK;
}

static tmd_status launch_network(const DevModel &dm, const int32_t *perm, const int32_t *types, int64_t n,
                                 const float *G, float *dG, float *e_atom, double *part_e, int *ntile_out,
                                 cudaStream_t s) {
    tmd_status st;
    if (dm.precision == TMD_PREC_BF16 && network_kernel() != 2 && mlp_umma_supported(dm))
        return mlp_umma_launch(dm, perm, types, n, G, dG, e_atom, part_e, ntile_out, s);
    if (dm.precision == TMD_PREC_BF16 && network_kernel() == 1) {
        set_error("the tcgen05 network kernel does not support these network shapes");
        return TMD_ERR_UNIMPLEMENTED;
    }
    if ((st = set_mlp_smem(dm, dm.precision == TMD_PREC_BF16)) != TMD_OK) return st;
    if (dm.precision == TMD_PREC_BF16) {
        const int ntile = (int)((n + BT - 1) / BT);
        const BfCfg bcfg = mlp_bf16_cfg(dm);
        TMD_LAUNCH("k_mlp_bf16", s, k_mlp_bf16<<<ntile, BF_THREADS, mlp_bf16_smem_bytes(dm), s>>>(
                                        dm, perm, types, n, G, dG, e_atom, part_e, bcfg.bnc, bcfg.compact ? 1 : 0));
        *ntile_out = ntile;
    } else if (mlp_use_res(dm)) {
        static int per_sm = 0, nsm = 0;   // resident blocks of k_mlp_res per SM
        if (!per_sm) {
            const int smem = (int)(RW_SMEM_FLOATS * sizeof(float));
            TMD_CUDA(cudaFuncSetAttribute(k_mlp_res, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            int dev = 0;
            TMD_CUDA(cudaGetDevice(&dev));
            TMD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            TMD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_res, RW_THREADS, smem));
            per_sm = std::max(per_sm, 1);
        }
        const int64_t ntile = (n + RW_TR - 1) / RW_TR;
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntile, (int64_t)per_sm * nsm));
        TMD_LAUNCH("k_mlp_res", s, k_mlp_res<<<grid, RW_THREADS, RW_SMEM_FLOATS * sizeof(float), s>>>(
                                       dm, perm, types, n, G, dG, e_atom, part_e));
        *ntile_out = (int)ntile;
    } else {
        const int tr = mlp_tr(dm);
        const int ntile = (int)((n + tr - 1) / tr);
        if (tr == 64)
            TMD_LAUNCH("k_mlp", s, k_mlp<64><<<ntile, MLP_THREADS, mlp_smem_bytes(dm), s>>>(dm, perm, types, n, G, dG,
                                                                                             e_atom, part_e));
        else
            TMD_LAUNCH("k_mlp", s, k_mlp<32><<<ntile, MLP_THREADS, mlp_smem_bytes(dm), s>>>(dm, perm, types, n, G, dG,
                                                                                             e_atom, part_e));
        *ntile_out = ntile;
    }
    TMD_CUDA(cudaGetLastError());
    return TMD_OK;
}

static tmd_status split_positions(tmd_nlist *nl, const double *pos, int64_t n, cudaStream_t s) {
    tmd_status st;
    if ((st = grow(&nl->ph, &nl->cap_ph, n)) != TMD_OK) return st;
    if ((st = grow(&nl->pl, &nl->cap_pl, n)) != TMD_OK) return st;
    TMD_LAUNCH("k_split_pos", s, k_split_pos<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, n, nl->ph, nl->pl));
    TMD_CUDA(cudaGetLastError());
    return TMD_OK;
}

// room for the in-cutoff pair cache: one slot per table entry, a count per atom
static tmd_status pair_cache(tmd_nlist *nl, int64_t n_atoms, cudaStream_t) {
    tmd_status st;
    const int64_t cap = std::max<int64_t>(nl->nnz, 1);
    if ((st = grow(&nl->pq, &nl->cap_pq, cap)) != TMD_OK) return st;
    if ((st = grow(&nl->pq2, &nl->cap_pq2, cap)) != TMD_OK) return st;
    return grow(&nl->npair, &nl->cap_npair, std::max<int64_t>(n_atoms, 1));
}

// Every workspace an evaluation of n_active atoms (arrays of n_total atoms)
// uses, sized before any launch: a captured launch sequence must find them
// already in place.
tmd_status reserve_compute(const DevModel &dm, tmd_nlist *nl, int64_t n_total, int64_t n_active) {
    tmd_status st;
    const int64_t nt = std::max<int64_t>(n_total, 1), na = std::max<int64_t>(n_active, 1);
    if ((st = grow(&nl->G, &nl->cap_G, na * dm.Dd)) != TMD_OK) return st;
    if ((st = grow(&nl->dG, &nl->cap_dG, na * dm.Dd)) != TMD_OK) return st;
    if ((st = grow(&nl->P, &nl->cap_P, na * dm.S * dm.K * NMOM)) != TMD_OK) return st;
    if ((st = grow(&nl->Fq, &nl->cap_Fq, 3 * nt)) != TMD_OK) return st;
    if ((st = grow(&nl->ph, &nl->cap_ph, nt)) != TMD_OK) return st;
    if ((st = grow(&nl->pl, &nl->cap_pl, nt)) != TMD_OK) return st;
    const int64_t nblk = pair_blocks(dm, na), ntile = (na + MT - 1) / MT;
    if ((st = grow(&nl->part, &nl->cap_part, ntile + 9 * nblk + 16 + RED_PART)) != TMD_OK) return st;
    return pair_cache(nl, nt, nullptr);
}

static DevNlist dev_nlist(const tmd_nlist *nl, int64_t n, const double box[3]) {
    DevNlist dn;
    dn.beg = nl->beg;
    dn.end = nl->end;
    dn.nbr = nl->nbr;
    dn.shift = nl->shift;
    dn.perm = nl->perm;
    dn.ph = nl->ph;
    dn.pl = nl->pl;
    dn.n = n;
    for (int x = 0; x < 3; ++x) {
        dn.box[x] = box[x];
        grid_split(box[x], dn.Lh[x], dn.Ll[x]);
    }
    return dn;
}

tmd_status run_descriptors(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                           int64_t n, const double box[3], float *G, float *dEdG, cudaStream_t s) {
    tmd_status st = validate(model, nl, n, box);
    if (st != TMD_OK) return st;
    if (n == 0) return TMD_OK;
    const DevModel &dm = model->dm;
    if ((st = grow(&nl->P, &nl->cap_P, n * dm.S * dm.K * NMOM)) != TMD_OK) return st;
    if ((st = grow(&nl->G, &nl->cap_G, n * dm.Dd)) != TMD_OK) return st;
    if (dEdG && (st = grow(&nl->dG, &nl->cap_dG, n * dm.Dd)) != TMD_OK) return st;
    const int nblk = pair_blocks(dm, n);
    if ((st = split_positions(nl, pos, n, s)) != TMD_OK) return st;
    const DevNlist dn = dev_nlist(nl, n, box);
    if ((st = dispatch_pair(dm, dn, pos, types, nl, nullptr, nblk, s, true)) != TMD_OK) return st;
    // the workspaces hold rows in perm order; the caller's arrays are per atom
    const unsigned gb = (unsigned)std::min<int64_t>((n * dm.Dd / 4 + 255) / 256, 65535);
    TMD_LAUNCH("k_rows_to_atoms", s, k_rows_to_atoms<<<gb, 256, 0, s>>>(nl->G, nl->perm, n, dm.Dd, G));
    TMD_CUDA(cudaGetLastError());
    if (!dEdG) return TMD_OK;
    const int ntile = (int)((n + MT - 1) / MT);
    if ((st = grow(&nl->part, &nl->cap_part, ntile + 16)) != TMD_OK) return st;
    int nt = 0;
    if ((st = launch_network(dm, nl->perm, types, n, nl->G, nl->dG, nullptr, nl->part, &nt, s)) != TMD_OK) return st;
    TMD_LAUNCH("k_rows_to_atoms", s, k_rows_to_atoms<<<gb, 256, 0, s>>>(nl->dG, nl->perm, n, dm.Dd, dEdG));
    TMD_CUDA(cudaGetLastError());
    return TMD_OK;
}

tmd_status run_compute(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types, int64_t n,
                       const double box[3], double *energy, float *e_atom, float *forces, double *virial,
                       cudaStream_t s, bool pos_split) {
    tmd_status st0 = validate(model, nl, n, box);
    if (st0 != TMD_OK) return st0;
    const DevModel &dm = model->dm;
    if (n == 0) {
        if (energy) TMD_CUDA(cudaMemsetAsync(energy, 0, sizeof(double), s));
        if (virial) TMD_CUDA(cudaMemsetAsync(virial, 0, 9 * sizeof(double), s));
        return TMD_OK;
    }
    tmd_status st;
    const int64_t Dd = dm.Dd;
    if ((st = grow(&nl->G, &nl->cap_G, n * Dd)) != TMD_OK) return st;
    if ((st = grow(&nl->dG, &nl->cap_dG, n * Dd)) != TMD_OK) return st;
    if ((st = grow(&nl->P, &nl->cap_P, n * dm.S * dm.K * NMOM)) != TMD_OK) return st;
    if ((st = grow(&nl->Fq, &nl->cap_Fq, 3 * n)) != TMD_OK) return st;
    const int nblk = pair_blocks(dm, n);
    const int ntile = (int)((n + MT - 1) / MT);
    if ((st = grow(&nl->part, &nl->cap_part, ntile + 9 * (int64_t)nblk + 16 + RED_PART)) != TMD_OK) return st;
    double *part_e = nl->part;
    double *part_w = nl->part + ntile;

    if (!(pos_split && nl->cap_ph >= n && nl->cap_pl >= n))
        if ((st = split_positions(nl, pos, n, s)) != TMD_OK) return st;
    if ((st = pair_cache(nl, n, s)) != TMD_OK) return st;
    DevNlist dn = dev_nlist(nl, n, box);
    dn.pq = nl->pq;
    dn.pq2 = nl->pq2;
    dn.npair = nl->npair;

    TMD_CUDA(cudaMemsetAsync(nl->Fq, 0, sizeof(long long) * 3 * n, s));
    if ((st = dispatch_pair(dm, dn, pos, types, nl, part_w, nblk, s, true)) != TMD_OK) return st;
    int ne = 0;
    if ((st = launch_network(dm, nl->perm, types, n, nl->G, nl->dG, e_atom, part_e, &ne, s)) != TMD_OK) return st;
    if ((st = dispatch_pair(dm, dn, pos, types, nl, part_w, nblk, s, false)) != TMD_OK) return st;
    TMD_LAUNCH("k_reduce", s, k_reduce_part<<<RED_BLOCKS, 256, 0, s>>>(part_e, ne, part_w, nblk, part_w + 9 * (size_t)nblk + 16));
    TMD_LAUNCH("k_reduce", s, k_reduce<<<1, 32, 0, s>>>(part_w + 9 * (size_t)nblk + 16, energy, virial));
    TMD_CUDA(cudaGetLastError());
    if (forces) {
        TMD_LAUNCH("k_forces_out", s, k_forces_out<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(
                                           reinterpret_cast<const long long *>(nl->Fq), n, forces));
        TMD_CUDA(cudaGetLastError());
    }
    return TMD_OK;
}

// owned atoms [0, n_owned) per species
__global__ void k_count_species(const int32_t *__restrict__ types, int64_t n_owned, int32_t *__restrict__ count) {
    __shared__ int32_t c[TMD_MAX_SPECIES];
    if (threadIdx.x < TMD_MAX_SPECIES) c[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_owned; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&c[types[i]], 1);
    __syncthreads();
    if (threadIdx.x < TMD_MAX_SPECIES) atomicAdd(&count[threadIdx.x], c[threadIdx.x]);
}

// The centres are the owned atoms [0, n_owned); atoms [n_owned, n) are ghosts
// (copies of other domains' atoms within the list radius of this one): they
// are neighbours of the centres, hold no energy term of their own, and
// receive their share of the pair forces, which the caller hands back to the
// domains that own them.  The table's perm groups atoms by species in index
// order, so the owned atoms of species t are the first owned-count[t] of
// block t.
tmd_status run_compute_owned(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                             int64_t n, int64_t n_owned, const double box[3], double *energy, float *e_atom,
                             float *forces, double *virial, cudaStream_t s) {
    tmd_status st = validate(model, nl, n, box);
    if (st != TMD_OK) return st;
    if (n_owned < 0 || n_owned > n) {
        set_error("n_owned = %lld outside [0, %lld]", (long long)n_owned, (long long)n);
        return TMD_ERR_INVALID_ARG;
    }
    if (n_owned == n) return run_compute(model, nl, pos, types, n, box, energy, e_atom, forces, virial, s);
    const DevModel &dm = model->dm;
    if ((st = grow(&nl->own_count, &nl->cap_own_count, TMD_MAX_SPECIES)) != TMD_OK) return st;
    if ((st = grow(&nl->perm_own, &nl->cap_perm_own, std::max<int64_t>(n_owned, 1))) != TMD_OK) return st;
    TMD_CUDA(cudaMemsetAsync(nl->own_count, 0, sizeof(int32_t) * TMD_MAX_SPECIES, s));
    if (n_owned > 0)
        TMD_LAUNCH("k_count_species", s, k_count_species<<<(unsigned)std::min<int64_t>((n_owned + 255) / 256, 1024), 256, 0,
                                                           s>>>(types, n_owned, nl->own_count));
    TMD_CUDA(cudaGetLastError());
    int32_t own[TMD_MAX_SPECIES];
    TMD_CUDA(cudaMemcpyAsync(own, nl->own_count, sizeof(own), cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaStreamSynchronize(s));
    int64_t src = 0, dst = 0;
    for (int t = 0; t < TMD_MAX_SPECIES; ++t) {
        if (own[t] > 0)
            TMD_CUDA(cudaMemcpyAsync(nl->perm_own + dst, nl->perm + src, sizeof(int32_t) * own[t],
                                     cudaMemcpyDeviceToDevice, s));
        dst += own[t];
        src += nl->type_count[t];
    }
    if (dst != n_owned) {
        set_error("owned atoms per species do not add up to n_owned");
        return TMD_ERR_INVALID_ARG;
    }
    if (e_atom) TMD_CUDA(cudaMemsetAsync(e_atom, 0, sizeof(float) * n, s));
    if (n_owned == 0) {
        if (energy) TMD_CUDA(cudaMemsetAsync(energy, 0, sizeof(double), s));
        if (virial) TMD_CUDA(cudaMemsetAsync(virial, 0, 9 * sizeof(double), s));
        if (forces) TMD_CUDA(cudaMemsetAsync(forces, 0, sizeof(float) * 3 * n, s));
        return TMD_OK;
    }
    if ((st = reserve_compute(dm, nl, n, n_owned)) != TMD_OK) return st;
    const int nblk = pair_blocks(dm, n_owned);
    const int ntile = (int)((n_owned + MT - 1) / MT);
    double *part_e = nl->part;
    double *part_w = nl->part + ntile;
    if ((st = split_positions(nl, pos, n, s)) != TMD_OK) return st;
    DevNlist dn = dev_nlist(nl, n_owned, box);
    dn.perm = nl->perm_own;
    dn.pq = nl->pq;
    dn.pq2 = nl->pq2;
    dn.npair = nl->npair;
    TMD_CUDA(cudaMemsetAsync(nl->Fq, 0, sizeof(long long) * 3 * n, s));
    if ((st = dispatch_pair(dm, dn, pos, types, nl, part_w, nblk, s, true)) != TMD_OK) return st;
    int ne = 0;
    if ((st = launch_network(dm, nl->perm_own, types, n_owned, nl->G, nl->dG, e_atom, part_e, &ne, s)) != TMD_OK)
        return st;
    if ((st = dispatch_pair(dm, dn, pos, types, nl, part_w, nblk, s, false)) != TMD_OK) return st;
    TMD_LAUNCH("k_reduce", s, k_reduce_part<<<RED_BLOCKS, 256, 0, s>>>(part_e, ne, part_w, nblk, part_w + 9 * (size_t)nblk + 16));
    TMD_LAUNCH("k_reduce", s, k_reduce<<<1, 32, 0, s>>>(part_w + 9 * (size_t)nblk + 16, energy, virial));
    TMD_CUDA(cudaGetLastError());
    if (forces) {
        TMD_LAUNCH("k_forces_out", s, k_forces_out<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(
                                           reinterpret_cast<const long long *>(nl->Fq), n, forces));
        TMD_CUDA(cudaGetLastError());
    }
    return TMD_OK;
}

}  // namespace tmd

// ---------------------------------------------------------------------------
// Allocation-free force evaluation (tmd_compute_noalloc).
//
// For callers that cannot allocate device memory while they run: codes that
// hand all GPU memory to their own pool allocator up front, or that must not
// pay for or synchronise on an allocation inside their time-stepping loop.
// The caller passes the neighbour table and every input and output; all
// scratch (position split, identity atom order, P, G, G', fixed-point force
// accumulator, block partials) lives in one static device array, which every
// GPU that loads the library holds until the process exits.
// ---------------------------------------------------------------------------
namespace tmd {

namespace {

constexpr size_t NOALLOC_BYTES = size_t(64) << 20;  // 64 MiB of scratch per device
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[256] = {nullptr};

__global__ void k_iota(int32_t *__restrict__ perm, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (int32_t)i;
}

// Checks the caller's table and species (the kernels index per-species
// tables with them) and records a violation in *flag.
__global__ void k_noalloc_check(const int64_t *__restrict__ off, const int32_t *__restrict__ nbr,
                                const char4 *__restrict__ shift, const int32_t *__restrict__ types, int64_t n,
                                int64_t nnz, int S, double Lx, double Ly, double Lz, int32_t *__restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0 && (off[0] != 0 || off[n] != nnz)) atomicOr(flag, 1);
    for (int64_t i = t0; i < n; i += stride) {
        if (off[i + 1] < off[i]) atomicOr(flag, 1);
        if (types[i] < 0 || types[i] >= S) atomicOr(flag, 2);
    }
    for (int64_t c = t0; c < nnz; c += stride) {
        const int j = nbr[c];
        const int b = shift[c].w;
        if (j < 0 || j >= n) atomicOr(flag, 4);
        else if (b != types[j]) atomicOr(flag, 16);   // the species byte must be that of j
        if (b < 0 || b >= S) atomicOr(flag, 8);
        const char4 sh = shift[c];   // the pair geometry keeps |s| L below the grid limit
        if (abs((int)sh.x) * Lx >= GRID_LIMIT / 2 || abs((int)sh.y) * Ly >= GRID_LIMIT / 2 ||
            abs((int)sh.z) * Lz >= GRID_LIMIT / 2)
            atomicOr(flag, 32);
    }
}

}  // namespace

tmd_status noalloc_capacity(const tmd_model *model, int64_t n, size_t *need) {
    const DevModel &dm = model->dm;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const int64_t nblk = (int64_t)pair_blocks(dm, n);
    const int64_t ntile = (n + MT - 1) / MT;
    size_t b = 0;
    b += al(sizeof(int32_t) * n);                              // identity order
    b += 2 * al(sizeof(float4) * n);                           // positions hi / lo
    b += al(sizeof(float) * n * dm.S * dm.K * NMOM);           // P
    b += 2 * al(sizeof(float) * n * dm.Dd);                    // G, G'
    b += al(sizeof(unsigned long long) * 3 * n);               // force accumulator
    b += al(sizeof(double) * (ntile + 9 * nblk + 16 + RED_PART));         // block partials
    b += al(sizeof(int32_t) * 4);                              // check flag
    *need = b;
    return b <= NOALLOC_BYTES ? TMD_OK : TMD_ERR_CAPACITY;
}

tmd_status run_compute_noalloc(const tmd_model *model, const int64_t *off, const int32_t *nbr, const int8_t *shift4,
                               int64_t nnz, const double *pos, const int32_t *types, int64_t n, const double box[3],
                               double *energy, float *e_atom, float *forces, double *virial, cudaStream_t s) {
    if (!model || !box) {
        set_error("null model or box");
        return TMD_ERR_INVALID_ARG;
    }
    if (n < 0 || n >= (int64_t(1) << 28) || nnz < 0) {
        set_error("n = %lld or nnz = %lld out of range", (long long)n, (long long)nnz);
        return TMD_ERR_INVALID_ARG;
    }
    for (int x = 0; x < 3; ++x)
        if (!(std::isfinite(box[x]) && box[x] > 0.0 && box[x] < GRID_LIMIT / 2)) {
            set_error("box[%d] must be finite, > 0 and below %.0f A", x, GRID_LIMIT / 2);
            return TMD_ERR_INVALID_ARG;
        }
    if (n > 0 && (!off || !pos || !types || (nnz > 0 && (!nbr || !shift4)))) {
        set_error("null off/nbr/shift4/pos/types");
        return TMD_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(shift4) & 3) != 0) {
        set_error("shift4 must be 4-byte aligned");
        return TMD_ERR_INVALID_ARG;
    }
    size_t need = 0;
    if (noalloc_capacity(model, n, &need) != TMD_OK) {
        set_error("%lld atoms need %zu bytes of scratch; the static scratch holds %zu", (long long)n, need,
                  NOALLOC_BYTES);
        return TMD_ERR_CAPACITY;
    }
    int dev = 0;
    TMD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("device ordinal %d out of range", dev);
        return TMD_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    {
        // once per device, with that device current: the host-side name of a
        // __device__ array is not a device address; ask the runtime for it.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            TMD_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_addr[dev] = p;
        }
        base = g_noalloc_addr[dev];
    }
    const DevModel &dm = model->dm;
    if (n == 0) {
        if (energy) TMD_CUDA(cudaMemsetAsync(energy, 0, sizeof(double), s));
        if (virial) TMD_CUDA(cudaMemsetAsync(virial, 0, 9 * sizeof(double), s));
        return TMD_OK;
    }
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    unsigned char *cur = static_cast<unsigned char *>(base);
    auto take = [&](size_t bytes) {
        void *p = cur;
        cur += al(bytes);
        return p;
    };
    const int nblk = pair_blocks(dm, n);
    const int ntile = (int)((n + MT - 1) / MT);
    tmd_nlist w;  // a view onto the static scratch; never freed
    w.perm = static_cast<int32_t *>(take(sizeof(int32_t) * n));
    w.ph = static_cast<float4 *>(take(sizeof(float4) * n));
    w.pl = static_cast<float4 *>(take(sizeof(float4) * n));
    w.P = static_cast<float *>(take(sizeof(float) * n * dm.S * dm.K * NMOM));
    w.G = static_cast<float *>(take(sizeof(float) * n * dm.Dd));
    w.dG = static_cast<float *>(take(sizeof(float) * n * dm.Dd));
    w.Fq = static_cast<unsigned long long *>(take(sizeof(unsigned long long) * 3 * n));
    w.part = static_cast<double *>(take(sizeof(double) * (ntile + 9 * (size_t)nblk + 16 + RED_PART)));
    int32_t *flag = static_cast<int32_t *>(take(sizeof(int32_t) * 4));

    // validate the caller's table on the device, then read the result
    TMD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    const int cb = (int)std::min<int64_t>((std::max(n, nnz) + 255) / 256, 4096);
    TMD_LAUNCH("k_noalloc_check", s, k_noalloc_check<<<cb, 256, 0, s>>>(off, nbr, reinterpret_cast<const char4 *>(shift4),
                                                                        types, n, nnz, dm.S, box[0], box[1], box[2],
                                                                        flag));
    TMD_CUDA(cudaGetLastError());
    int32_t bad = 0;
    TMD_CUDA(cudaMemcpyAsync(&bad, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaStreamSynchronize(s));
    if (bad) {
        set_error("invalid neighbour table or species (check code %d: 1 offsets, 2 types, 4 nbr ids, 8 shift4 species "
                  "out of range, 16 shift4 species differs from types[nbr], 32 |shift| box >= 4096 A)",
                  bad);
        return TMD_ERR_INVALID_ARG;
    }

    TMD_LAUNCH("k_iota", s, k_iota<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.perm, n));
    TMD_LAUNCH("k_split_pos", s, k_split_pos<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, n, w.ph, w.pl));
    TMD_CUDA(cudaGetLastError());
    DevNlist dn;
    dn.beg = off;        // CSR: the segment of atom a is [off[a], off[a + 1])
    dn.end = off + 1;
    dn.nbr = nbr;
    dn.shift = reinterpret_cast<const char4 *>(shift4);
    dn.perm = w.perm;
    dn.ph = w.ph;
    dn.pl = w.pl;
    dn.n = n;
    for (int x = 0; x < 3; ++x) {
        dn.box[x] = box[x];
        grid_split(box[x], dn.Lh[x], dn.Ll[x]);
    }
    double *part_e = w.part;
    double *part_w = w.part + ntile;
    tmd_status st;
    // the accumulator keeps the previous call's contents: clear it
    TMD_CUDA(cudaMemsetAsync(w.Fq, 0, sizeof(unsigned long long) * 3 * n, s));
    if ((st = dispatch_pair(dm, dn, pos, types, &w, part_w, nblk, s, true)) != TMD_OK) return st;
    int ne = 0;
    if ((st = launch_network(dm, w.perm, types, n, w.G, w.dG, e_atom, part_e, &ne, s)) != TMD_OK) return st;
    if ((st = dispatch_pair(dm, dn, pos, types, &w, part_w, nblk, s, false)) != TMD_OK) return st;
    TMD_LAUNCH("k_reduce", s, k_reduce_part<<<RED_BLOCKS, 256, 0, s>>>(part_e, ne, part_w, nblk, part_w + 9 * (size_t)nblk + 16));
    TMD_LAUNCH("k_reduce", s, k_reduce<<<1, 32, 0, s>>>(part_w + 9 * (size_t)nblk + 16, energy, virial));
    TMD_CUDA(cudaGetLastError());
    if (forces) {
        TMD_LAUNCH("k_forces_out", s, k_forces_out<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(
                                           reinterpret_cast<const long long *>(w.Fq), n, forces));
        TMD_CUDA(cudaGetLastError());
    }
    return TMD_OK;
}

}  // namespace tmd

namespace tmd {

void sys_reduce_launch(const int32_t *act, int n_act, const int64_t *off, const float *e_atom, const float *w_atom,
                       const double *vel, const double *mass, double *out, cudaStream_t s) {
    k_sys_reduce<<<n_act, 256, 0, s>>>(act, off, e_atom, w_atom, vel, mass, out);
}

tmd_status run_compute_batch(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                             int64_t n_total, const int32_t *sys_of, float *forces, float *e_atom, float *w_atom,
                             const int32_t *act_list, int n_act, const int64_t *sys_off, const double *vel,
                             const double *mass, double *sys_out, cudaStream_t s) {
    if (!model || !nl || !nl->built) {
        set_error("null model or table not built");
        return TMD_ERR_INVALID_ARG;
    }
    const DevModel &dm = model->dm;
    for (int t = dm.S; t < TMD_MAX_SPECIES; ++t)
        if (nl->type_count[t] != 0) {
            set_error("species id %d present but the model has %d species", t, dm.S);
            return TMD_ERR_INVALID_ARG;
        }
    const int64_t na = nl->n_active;  // atoms of the active systems, in perm
    tmd_status st;
    if (na > 0) {
        // P, G and G' are indexed by perm position: room for the active atoms only
        if ((st = grow(&nl->G, &nl->cap_G, na * dm.Dd)) != TMD_OK) return st;
        if ((st = grow(&nl->dG, &nl->cap_dG, na * dm.Dd)) != TMD_OK) return st;
        if ((st = grow(&nl->P, &nl->cap_P, na * dm.S * dm.K * NMOM)) != TMD_OK) return st;
        if ((st = grow(&nl->Fq, &nl->cap_Fq, 3 * n_total)) != TMD_OK) return st;
        const int nblk = pair_blocks(dm, na);
        const int ntile = (int)((na + MT - 1) / MT);
        if ((st = grow(&nl->part, &nl->cap_part, ntile + 9 * (int64_t)nblk + 16 + RED_PART)) != TMD_OK) return st;
        if ((st = split_positions(nl, pos, n_total, s)) != TMD_OK) return st;
        if ((st = pair_cache(nl, n_total, s)) != TMD_OK) return st;
        DevNlist dn = dev_nlist(nl, na, nl->box);
        dn.sp = nl->sp;
        dn.sys_of = sys_of;
        dn.pq = nl->pq;
        dn.pq2 = nl->pq2;
        dn.npair = nl->npair;
        TMD_CUDA(cudaMemsetAsync(nl->Fq, 0, sizeof(long long) * 3 * n_total, s));
        if ((st = dispatch_pair(dm, dn, pos, types, nl, nullptr, nblk, s, true)) != TMD_OK) return st;
        int ne = 0;
        if ((st = launch_network(dm, nl->perm, types, na, nl->G, nl->dG, e_atom, nl->part, &ne, s)) != TMD_OK)
            return st;
        if ((st = dispatch_pair(dm, dn, pos, types, nl, nl->part + ntile, nblk, s, false, w_atom)) != TMD_OK)
            return st;
        TMD_LAUNCH("k_forces_out_perm", s, k_forces_out_perm<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(
                                               reinterpret_cast<const long long *>(nl->Fq), nl->perm, na, forces));
        TMD_CUDA(cudaGetLastError());
    }
    if (n_act > 0) {
        TMD_LAUNCH("k_sys_reduce", s, k_sys_reduce<<<n_act, 256, 0, s>>>(act_list, sys_off, e_atom, w_atom, vel, mass,
                                                                         sys_out));
        TMD_CUDA(cudaGetLastError());
    }
    return TMD_OK;
}

}  // namespace tmd
