// BF16 network form on the fifth-generation tensor cores (tcgen05): the
// per-species atomic-energy network E_a = NNP(G_a) and its input gradient
// G' = dE_a/dG_a (Sec. "The Tensor Formalism", the E_a / NNP equations and
// the backward chain through the network), for 128-atom tiles.
//
// Every product of the chain -- forward layers a_{l+1} = act(a_l W_l^T + b_l),
// then dz_l = (dz_{l+1} W_l) * act'(a_l) down to G' = dz_1 W_0 -- is one
// [128 x K] x [K x N] tcgen05.mma GEMM with BF16 operands in shared memory and
// the FP32 accumulator in tensor memory (TMEM lane = tile row = atom).  The
// weight operand streams in 64-wide K chunks by bulk copy (cp.async.bulk,
// completion on an mbarrier) into a ring of two to four stages (resident when
// one species' whole chain fits); the first layer's operand is the FP32
// descriptor tile converted to BF16 by the threads, chunk by chunk.
// After each product eight warps read the accumulator back (tcgen05.ld, one
// row per thread; the two warps of a TMEM lane quarter take alternate
// 16-column blocks), apply bias and activation, keep act' in TMEM for the
// backward chain (tcgen05.st) and write the BF16 operand of the next product.
// One elected thread issues the MMAs and the copies.
//
// Operand layout (no swizzle, K-major): 8 x 8 BF16 core matrices of 128
// contiguous bytes; along K the next core matrix is 128 B away (LBO), the
// next group of 8 rows 1024 B away (SBO), i.e. a 64-wide K chunk of R rows is
// [R/8][8 core matrices][8 rows][8 elements].
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "net_common.cuh"
#include "tmd_internal.cuh"

namespace tmd {

// status bits of the tensor-core kernels (bounded waits that ran out)
__device__ int32_t g_umma_status = 0;

namespace {

constexpr int UM = 128;                 // atoms per tile: the MMA M, one TMEM lane each
constexpr int UTHREADS = 256;           // 8 warps; warp w owns TMEM lanes / rows 32 (w % 4) .. + 31 and
                                        // the 16-column blocks b of each epilogue with b % 2 == w / 4
constexpr int UKC = 64;                 // K per streamed chunk
constexpr int UNMAX = 256;              // largest N of one MMA
constexpr uint32_t WAIT_LIMIT = 1u << 22;
constexpr int CHUNK_EL = UM * UKC;      // elements of a 128-row K chunk

struct UmmaNet {
    int xchunks;        // 64-wide K chunks of an activation buffer (widest hidden layer)
    int np_max;         // largest MMA N of any product
    int npass0, np0;    // N passes of the last product (G') and their width
    int tcols;          // TMEM columns allocated per block
    int dercol[MAX_LAYERS];   // TMEM column of act'(a_l), l = 1 .. L-1
    int smem;           // dynamic shared memory bytes
    int blocks_per_sm;
    int nst;            // weight-chunk stages (2 .. MAX_NST)
    int block_chunks;   // weight chunks of one species block (all products)
    int resident;       // one species whose chunks all fit the stages: copied once per block
    int alias;          // one K chunk in the first layer: its G stage is also activation buffer X0
    int cstride;        // floats per species of the staged constants: biases, w_out, b_out
    int cbias[MAX_LAYERS + 1];   // offset of the bias of layer l (l < L), of w_out (l = L), of b_out (l = L + 1)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr uint64_t WAIT_NS = 200000000ull;   // 0.2 s per wait

// Bounded wait for the completion of the phase with this parity.  When it
// gives up (0.2 s, or the iteration cap) it records DEV_ERR_TIMEOUT and sets
// the block's abort flag, after which every later wait returns at once: the
// kernel runs on to its end, waits (bounded) for its copies and MMAs in
// flight, frees its tensor memory and the host reports the status; the
// results of that call are not valid.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort) {
    if (*abort) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 1; i < WAIT_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0 && (*abort || gtimer() - t0 > WAIT_NS)) break;
    }
    *abort = 1;
    atomicOr(&g_umma_status, DEV_ERR_TIMEOUT);
    return false;
}
// teardown after an abort: wait, bounded, for a phase regardless of the flag
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = gtimer();
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity) || ((i & 63) == 0 && gtimer() - t0 > WAIT_NS)) return;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start address, LBO 128 B, SBO 1024 B,
// descriptor version 1 (bits 46-48), base offset 0, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor of kind::f16: D FP32 (bits 4-5), A BF16 (7-9),
// B BF16 (10-12), A and B K-major (bits 15, 16 clear), N >> 3 (17-22),
// M >> 4 (24-28)
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    // the registers are read only after the wait (tied through the asm operands)
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st16_nowait(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// element (row, k) of a chunked operand buffer, in elements from its start
__device__ __forceinline__ int op_index(int row, int k) {
    return (k / UKC) * CHUNK_EL + (row >> 3) * 512 + ((k % UKC) >> 3) * 64 + (row & 7) * 8 + (k & 7);
}
// 16 values as BF16 at (row, col0 .. col0 + 15), col0 a multiple of 16
__device__ __forceinline__ void store_row16(uint16_t *X, int row, int col0, const float (&v)[16]) {
    uint4 lo, hi;
    lo.x = pack_bf16(v[0], v[1]);
    lo.y = pack_bf16(v[2], v[3]);
    lo.z = pack_bf16(v[4], v[5]);
    lo.w = pack_bf16(v[6], v[7]);
    hi.x = pack_bf16(v[8], v[9]);
    hi.y = pack_bf16(v[10], v[11]);
    hi.z = pack_bf16(v[12], v[13]);
    hi.w = pack_bf16(v[14], v[15]);
    const int i = op_index(row, col0);
    *reinterpret_cast<uint4 *>(X + i) = lo;
    *reinterpret_cast<uint4 *>(X + i + 64) = hi;   // next core matrix along K
}

constexpr int MAX_NST = 4;   // weight-chunk stages at most
constexpr int MAX_CHUNKS = 64;   // weight chunks of one species block at most

__global__ void __launch_bounds__(UTHREADS, 2)
    k_mlp_umma(DevModel m, UmmaNet u, const int32_t *__restrict__ perm, const int32_t *__restrict__ types, int64_t n,
               const float *__restrict__ G, float *__restrict__ dG, float *__restrict__ e_atom,
               double *__restrict__ part_e, int ntile) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    // barriers: full[MAX_NST], empty[MAX_NST] (weight stages), aempty[2] (G stages), done
    __shared__ __align__(8) uint64_t s_bar[2 * MAX_NST + 3];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ int s_atom[UM], s_type[UM], s_range[2];
    __shared__ float s_e[2][UM], s_ep[2][UM];   // s_e: E_a of the rows, by tile parity
    // per product pr: (K, N, N of a pass, npass | nkc << 8 | layer << 16) and
    // (bias offset, TMEM column of the act' written (forward) or read
    // (backward), w_out offset, b_out offset); per weight chunk of a species
    // block: (element offset in ub[s], bytes)
    __shared__ int4 s_pa[2 * MAX_LAYERS], s_pb[2 * MAX_LAYERS];
    __shared__ int2 s_ck[MAX_CHUNKS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rq = warp & 3, ch = warp >> 2;   // TMEM lane quarter, column-block parity
    const int row = rq * 32 + lane;            // this thread's tile row
    const int L = m.L, Dd = m.Dd, NST = u.nst;
    // dynamic shared memory: X[2] activation buffers, 2 G stages, NST weight stages
    // (alias: the first layer has one K chunk, so the single G stage is also
    // the first activation buffer -- each use of it is ordered by the
    // product-completion waits)
    const int na = u.alias ? 1 : 2;   // G stages
    uint16_t *const X0 = reinterpret_cast<uint16_t *>(smraw);
    uint16_t *const X1 = X0 + (size_t)(u.alias ? max(u.xchunks, 1) : u.xchunks) * CHUNK_EL;
    uint16_t *const A0 = u.alias ? X0 : X1 + (size_t)u.xchunks * CHUNK_EL;
    uint16_t *const B0 = u.alias ? X1 + (size_t)u.xchunks * CHUNK_EL : A0 + 2 * CHUNK_EL;
    const size_t bstride = (size_t)u.np_max * UKC;   // elements per weight stage
    // biases, w_out and b_out of every species (read by every epilogue)
    float *const sconst = reinterpret_cast<float *>(B0 + (size_t)NST * bstride);
    for (int sp = 0; sp < m.S; ++sp)
        for (int i = tid; i < u.cstride; i += UTHREADS) {
            float v = 0.f;
            int l = 0;
            while (l <= L && i >= u.cbias[l + 1]) ++l;   // the part i falls in
            const int j = i - u.cbias[l];
            if (l < L) {
                if (j < m.dims[l + 1]) v = m.wf[sp][m.off_f[l] + (size_t)m.dims[l] * m.dims[l + 1] + j];
            } else if (l == L) {
                if (j < m.dims[L]) v = m.wb[sp][m.off_b[L] + j];
            } else if (j == 0) {
                v = m.wf[sp][m.off_f[L] + m.dims[L]];
            }
            sconst[sp * u.cstride + i] = v;
        }
    const uint32_t bar0 = smem_u32(&s_bar[0]);
    auto bar_full = [&](int st) { return bar0 + 8 * st; };
    auto bar_empty = [&](int st) { return bar0 + 8 * (MAX_NST + st); };
    auto bar_aempty = [&](int st) { return bar0 + 8 * (2 * MAX_NST + st); };
    const uint32_t bar_done = bar0 + 8 * (2 * MAX_NST + 2);
    if (tid == 0) {
        for (int i = 0; i < 2 * MAX_NST + 3; ++i) mbar_init(bar0 + 8 * i, 1);
        s_abort = 0;
        fence_proxy_async();
        int i = 0;
        for (int pr = 0; pr < 2 * L; ++pr) {
            const bool fwd = pr < L, last = pr == 2 * L - 1;
            const int l = fwd ? pr : 2 * L - 1 - pr;
            const int K = fwd ? m.dims[l] : m.dims[l + 1], N = fwd ? m.dims[l + 1] : m.dims[l];
            const int npass = last ? u.npass0 : 1, Np = last ? u.np0 : N, nkc = (K + UKC - 1) / UKC;
            s_pa[pr] = make_int4(K, N, Np, npass | nkc << 8 | l << 16);
            const int der = fwd ? (l < L - 1 ? u.dercol[l + 1] : 0) : (l >= 1 ? u.dercol[l] : 0);
            s_pb[pr] = make_int4(fwd ? u.cbias[l] : 0, der, u.cbias[L], u.cbias[L + 1]);
            for (int P = 0; P < npass; ++P)
                for (int c = 0; c < nkc; ++c, ++i)
                    s_ck[i] = make_int2(m.uoff[pr] + (P * nkc + c) * Np * UKC, Np * UKC * 2);
        }
    }
    volatile int *abort = &s_abort;
    uint32_t pending = 0;   // thread 0: stages with a copy not yet seen complete
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(u.tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t trow = tmem + ((uint32_t)(rq * 32) << 16);   // this warp's lane quarter, column 0
    uint32_t q = 0;    // weight chunks consumed
    int qs = 0;        // its stage, q % NST
    uint32_t qph = 0;  // the parity of its use, (q / NST) & 1
    uint32_t qi = 0;   // weight chunks whose copy was issued (thread 0)
    int qis = 0;       // its stage, qi % NST
    uint32_t qiu = 0;  // its use, qi / NST
    uint32_t ua = 0;   // G chunks consumed (stage ua & 1, use ua >> 1)
    uint32_t pd = 0;   // products (passes) completed
    // thread 0: issue the copies of this block's chunks up to global index lim
    auto issue_upto = [&](uint32_t lim, uint32_t qbase, int s) {
        if (u.resident && qi >= (uint32_t)NST) {   // the stages already hold every chunk
            qi = max(qi, lim);
            return;
        }
        while (qi < lim && !*abort) {
            const int st = qis;
            if (qiu >= 1) mbar_wait(bar_empty(st), (qiu - 1) & 1, abort);   // the MMAs that read it are done
            if (*abort) break;
            const int2 ck = s_ck[qi - qbase];
            mbar_expect_tx(bar_full(st), (uint32_t)ck.y);
            bulk_g2s(smem_u32(B0 + st * bstride), m.ub[s] + ck.x, (uint32_t)ck.y, bar_full(st));
            pending |= 1u << st;
            ++qi;
            if (++qis == NST) { qis = 0; ++qiu; }
        }
    };
    // Software pipeline over tiles: this thread's atom of the next tile, and
    // its share of that tile's first G chunk, are loaded into registers while
    // the current tile runs (a quarter warp per row: lane l covers row
    // 4 it + l / 8 of its lane quarter, columns 32 ch + 4 (l % 8) .. + 3 of
    // the chunk).
    auto row_atom = [&](int t) -> int {
        const int64_t p = (int64_t)t * UM + row;
        return (t < ntile && p < n) ? perm[p] : -1;
    };
    float4 gpre[8];
    uint32_t gok = 0;   // bit it: gpre[it] holds a row of an atom (else it reads as zeros)
    // G and G' rows are indexed by perm position: row r of tile t is t UM + r
    auto load_g0 = [&](int atom_of_my_row, int t) {
        gok = 0;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int a = __shfl_sync(0xffffffffu, atom_of_my_row, 4 * it + (lane >> 3));
            const int col = 32 * ch + 4 * (lane & 7);
            // the null row of a missing atom reads as zeros
            const bool ok = a >= 0 && col < Dd;
            const size_t p = (size_t)t * UM + rq * 32 + 4 * it + (lane >> 3);
            const float *src = G + (ok ? p * Dd + col : 0);
            float4 v;
            // issued here, in program order with the surrounding tensor-core
            // instructions, so that the loads overlap the rest of this tile
            asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                         : "l"(src));
            // raw registers: nothing here waits for the loads, the staging
            // of the next tile's first chunk does
            gpre[it] = v;
            gok |= (uint32_t)ok << it;
        }
    };
    // tile energy in FP64, fixed order (one warp): taken for the previous
    // tile while the current one waits on its first product
    auto tile_energy = [&](const float *e, int t) {
        double tsum = 0.0;
        for (int r = lane; r < UM; r += 32) tsum += (double)e[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
        if (lane == 0) part_e[t] = tsum;
    };
    constexpr int EWARP = UTHREADS / 32 - 1;   // the warp that sums (not the MMA issuer's)
    int kt = 0, prev_tile = -1;                // tiles done by this block, the last of them
    int nx_atom = row_atom(blockIdx.x);
    int nx_type = nx_atom >= 0 ? types[nx_atom] : -1;
    load_g0(nx_atom, blockIdx.x);
    for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int eb = kt & 1;
        if (ch == 0) {
            s_atom[row] = nx_atom;
            s_type[row] = nx_type;
            s_e[eb][row] = 0.f;
        }
        const int my_atom = nx_atom, my_type = nx_type;
        bool g0_ready = true;   // gpre holds this tile's first chunk
        // the tile after this one: atom ids now, species and G rows once gpre is consumed
        nx_atom = row_atom(tile + gridDim.x);
        __syncthreads();
        if (warp == 0) {   // species present in the tile (perm groups atoms by species)
            int lo = TMD_MAX_SPECIES, hi = -1;
            for (int r = lane; r < UM; r += 32)
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
        for (int s = s_lo; s <= s_hi; ++s) {
            const uint32_t qbase = q, qend = q + (uint32_t)u.block_chunks;
            if (tid == 0) issue_upto(min(qend, q + NST), qbase, s);
            for (int pr = 0; pr < 2 * L; ++pr) {
                const bool fwd = pr < L, last = pr == 2 * L - 1;
                const int4 pa = s_pa[pr], pb = s_pb[pr];
                const int K = pa.x, N = pa.y, Np = pa.z;
                const int npass = pa.w & 255, nkc = (pa.w >> 8) & 255, l = pa.w >> 16;   // l: layer of this product
                uint16_t *Xin = (pr & 1) ? X0 : X1, *Xout = (pr & 1) ? X1 : X0;
                for (int P = 0; P < npass; ++P) {
                    for (int c = 0; c < nkc; ++c) {
                        const int st = qs;
                        const int ast = ua & (na - 1);           // na is 1 or 2
                        const uint32_t ause = ua >> (na - 1);
                        uint16_t *Ast = A0 + ast * CHUNK_EL;
                        if (pr == 0) {   // G chunk c -> BF16 operand (a quarter warp per row, own rows)
                            if (!(c == 0 && g0_ready)) {
                                const int r0 = rq * 32 + (lane >> 3);
#pragma unroll
                                for (int it = 0; it < 8; ++it) {
                                    const int a = s_atom[r0 + 4 * it];
                                    const int col = c * UKC + 32 * ch + 4 * (lane & 7);
                                    gpre[it] = make_float4(0.f, 0.f, 0.f, 0.f);
                                    if (a >= 0 && col < Dd)
                                        gpre[it] = __ldg(reinterpret_cast<const float4 *>(
                                            G + ((size_t)tile * UM + r0 + 4 * it) * Dd + col));
                                }
                                gok = 0xffu;
                            }
                            if (ause >= 1) mbar_wait(bar_aempty(ast), (ause - 1) & 1, abort);
#pragma unroll
                            for (int it = 0; it < 8; ++it) {
                                const int r = rq * 32 + 4 * it + (lane >> 3);
                                const float4 gv = (gok >> it) & 1u ? gpre[it] : make_float4(0.f, 0.f, 0.f, 0.f);
                                uint2 w;
                                w.x = pack_bf16(gv.x, gv.y);
                                w.y = pack_bf16(gv.z, gv.w);
                                *reinterpret_cast<uint2 *>(Ast + op_index(r, 32 * ch + 4 * (lane & 7))) = w;
                            }
                            fence_proxy_async();
                            __syncthreads();
                        }
                        if (tid == 0 && !*abort) {
                            if (!(u.resident && q >= (uint32_t)NST) && mbar_wait(bar_full(st), qph, abort))
                                pending &= ~(1u << st);
                            tc_fence_after();
                            const int kl = min(UKC, K - c * UKC);
                            // the descriptors of the next K16 step are 256 bytes on (16 in the address field)
                            const uint64_t da = sdesc(smem_u32(pr == 0 ? Ast : Xin + (size_t)c * CHUNK_EL));
                            const uint64_t db = sdesc(smem_u32(B0 + st * bstride));
                            const uint32_t id = idesc_bf16(Np);
                            for (int j = 0; j < kl / 16; ++j)
                                umma_bf16(tmem, da + 16 * j, db + 16 * j, id, (c | j) != 0);
                            // resident weights: no copy ever waits for a stage to drain
                            if (!u.resident) umma_commit(bar_empty(st));
                            if (pr == 0) umma_commit(bar_aempty(ast));
                            // keep the stages filled: the copy for chunk q + NST - 1 reuses the
                            // stage of chunk q - 1, whose MMAs were issued one chunk earlier
                            issue_upto(min(qend, q + NST), qbase, s);
                        }
                        // the rest of warp 0 waits here rather than polling an
                        // mbarrier beside the issuing lane
                        if (warp == 0) __syncwarp();
                        if (pr == 0) {
                            // gpre is free: (re)start on the next tile's first chunk
                            // (after the MMA issue, which then waits on none of these loads)
                            if (g0_ready) nx_type = nx_atom >= 0 ? types[nx_atom] : -1;
                            g0_ready = false;
                            load_g0(nx_atom, tile + gridDim.x);
                            ++ua;
                        }
                        ++q;
                        if (++qs == NST) { qs = 0; qph ^= 1u; }
                    }
                    if (tid == 0) umma_commit(bar_done);
                    if (warp == 0) __syncwarp();
                    if (pr == 0 && P == 0 && s == s_lo && warp == EWARP && prev_tile >= 0)
                        tile_energy(s_e[eb ^ 1], prev_tile);
                    mbar_wait(bar_done, pd & 1, abort);
                    ++pd;
                    tc_fence_after();
                    // epilogue: this thread's row of the accumulator
                    if (fwd) {
                        const float *cs = sconst + s * u.cstride;
                        const float *bias = cs + pb.x;
                        const bool last_fwd = l == L - 1;
                        const float *wout = cs + pb.z;
                        float eacc = 0.f;
                        for (int c0 = 16 * ch; c0 < N; c0 += 32) {
                            float v[16], a[16], d[16];
                            tmem_ld16(trow + c0, v);
                            const float4 *b4 = reinterpret_cast<const float4 *>(bias + c0);
#pragma unroll
                            for (int e4 = 0; e4 < 4; ++e4) {
                                const float4 bb = b4[e4];
                                act_fd_bf16(m.act, v[4 * e4] + bb.x, m.sp_b, a[4 * e4], d[4 * e4]);
                                act_fd_bf16(m.act, v[4 * e4 + 1] + bb.y, m.sp_b, a[4 * e4 + 1], d[4 * e4 + 1]);
                                act_fd_bf16(m.act, v[4 * e4 + 2] + bb.z, m.sp_b, a[4 * e4 + 2], d[4 * e4 + 2]);
                                act_fd_bf16(m.act, v[4 * e4 + 3] + bb.w, m.sp_b, a[4 * e4 + 3], d[4 * e4 + 3]);
                            }
                            if (!last_fwd) {
                                store_row16(Xout, row, c0, a);
                                tmem_st16_nowait(trow + pb.y + c0, d);
                            } else {   // E_a partial and dz_L = w_out * act'(a_L)
                                const float4 *w4 = reinterpret_cast<const float4 *>(wout + c0);
#pragma unroll
                                for (int e4 = 0; e4 < 4; ++e4) {
                                    const float4 w = w4[e4];
                                    eacc = fmaf(w.x, a[4 * e4], eacc);
                                    eacc = fmaf(w.y, a[4 * e4 + 1], eacc);
                                    eacc = fmaf(w.z, a[4 * e4 + 2], eacc);
                                    eacc = fmaf(w.w, a[4 * e4 + 3], eacc);
                                    d[4 * e4] *= w.x;
                                    d[4 * e4 + 1] *= w.y;
                                    d[4 * e4 + 2] *= w.z;
                                    d[4 * e4 + 3] *= w.w;
                                }
                                store_row16(Xout, row, c0, d);
                            }
                        }
                        if (!last_fwd) tmem_st_wait();
                        if (last_fwd) s_ep[ch][row] = eacc;   // halves added after the product's barrier
                    } else if (!last) {   // dz_l = (dz_{l+1} W_l) * act'(a_l)
                        for (int c0 = 16 * ch; c0 < N; c0 += 32) {
                            float v[16], d[16];
                            tmem_ld16(trow + c0, v);
                            tmem_ld16(trow + pb.y + c0, d);
#pragma unroll
                            for (int e = 0; e < 16; ++e) v[e] *= d[e];
                            store_row16(Xout, row, c0, v);
                        }
                    } else {   // G' columns of this pass
                        // each warp's 32 x 16 blocks go out through shared memory
                        // (X1, unused during the last product) as 64-byte row
                        // pieces, four lanes to a row; the 16-byte groups of a
                        // staged row are permuted by bits 1-2 of the row so that
                        // both the row-wise writes and the transposed reads are
                        // free of bank conflicts
                        float *stg = reinterpret_cast<float *>(Xout) + warp * 512;
                        const int tc = lane & 3;
                        for (int c0 = 16 * ch; c0 < Np; c0 += 32) {
                            float v[16];
                            tmem_ld16(trow + c0, v);
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                *reinterpret_cast<float4 *>(stg + lane * 16 + 4 * (e ^ ((lane >> 1) & 3))) =
                                    make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
                            __syncwarp();
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int r = 8 * i + (lane >> 2);
                                const float4 w =
                                    *reinterpret_cast<const float4 *>(stg + r * 16 + 4 * (tc ^ ((r >> 1) & 3)));
                                if (s_type[rq * 32 + r] == s)
                                    *reinterpret_cast<float4 *>(dG + ((size_t)tile * UM + rq * 32 + r) * Dd + P * Np +
                                                                c0 + 4 * tc) = w;
                            }
                            __syncwarp();
                        }
                    }
                    fence_proxy_async();   // the operand writes are read by the next MMA
                    tc_fence_before();
                    __syncthreads();
                    if (pr == L - 1 && ch == 0 && my_type == s) {   // E_a of this species' rows
                        const float e = s_ep[0][row] + s_ep[1][row] + sconst[s * u.cstride + pb.w];
                        s_e[eb][row] = e;
                        if (e_atom) e_atom[my_atom] = e;
                    }
                }
            }
        }
        prev_tile = tile;
        ++kt;
    }
    __syncthreads();
    if (warp == EWARP && prev_tile >= 0) tile_energy(s_e[(kt - 1) & 1], prev_tile);
    if (tid == 0 && *abort) {   // bounded drain of this block's copies and MMAs in flight
        for (uint32_t k = (qi > (uint32_t)NST ? qi - NST : 0); k < qi; ++k)
            if (pending & (1u << (k % NST))) mbar_drain(bar_full(k % NST), (k / NST) & 1);
        umma_commit(bar_done);
        mbar_drain(bar_done, pd & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(u.tcols) : "memory");
}

// Self-test of the bounded waits: one warp allocates tensor memory, waits on
// an mbarrier that nothing signals, and must give up (about 0.2 s), record
// DEV_ERR_TIMEOUT, free its tensor memory and return.
__global__ void __launch_bounds__(32, 1) k_wait_probe(int32_t *__restrict__ gave_up) {
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const uint32_t bar = smem_u32(&s_bar);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        s_abort = 0;
        fence_proxy_async();
    }
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)), "r"(32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (threadIdx.x == 0) mbar_wait(bar, 0, &s_abort);   // nothing arrives: gives up
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
    if (threadIdx.x == 0) *gave_up = s_abort;
}

// launch plan for a model, or false when the shapes do not fit
int reg_blocks_per_sm();

bool plan(const DevModel &dm, UmmaNet &u) {
    const int reg_blocks = reg_blocks_per_sm();
    std::memset(&u, 0, sizeof(u));
    const int L = dm.L;
    for (int s = 0; s < dm.S; ++s)
        if (!dm.ub[s]) return false;
    int maxw = 0;
    for (int l = 0; l <= L; ++l)
        if (dm.dims[l] % 16) return false;
    for (int l = 1; l <= L; ++l) maxw = std::max(maxw, dm.dims[l]);
    if (maxw > UNMAX) return false;
    u.npass0 = (dm.Dd + UNMAX - 1) / UNMAX;
    if (dm.Dd % u.npass0) return false;
    u.np0 = dm.Dd / u.npass0;
    if (u.np0 % 16) return false;
    u.np_max = std::max(maxw, u.np0);
    u.xchunks = (maxw + UKC - 1) / UKC;
    // TMEM: accumulator columns [0, maxw), then act'(a_l) for l = 1 .. L-1;
    // the last product (G') may use every column (act' is dead by then)
    int col = maxw;
    for (int l = 1; l < L; ++l) {
        u.dercol[l] = col;
        col += dm.dims[l];
    }
    col = std::max(col, u.np0);
    if (col > 512) return false;
    u.tcols = 32;
    while (u.tcols < col) u.tcols <<= 1;
    u.block_chunks = 0;
    for (int pr = 0; pr < 2 * L; ++pr) {
        const bool fwd = pr < L;
        const int l = fwd ? pr : 2 * L - 1 - pr;
        const int K = fwd ? dm.dims[l] : dm.dims[l + 1];
        u.block_chunks += ((K + UKC - 1) / UKC) * (pr == 2 * L - 1 ? u.npass0 : 1);
    }
    if (u.block_chunks > MAX_CHUNKS) return false;
    // staged constants per species: bias of each layer, w_out, b_out
    int co = 0;
    for (int l = 0; l < L; ++l) {
        u.cbias[l] = co;
        co += dm.dims[l + 1];
    }
    u.cbias[L] = co;
    co += dm.dims[L];
    u.cbias[L + 1] = co;
    co += 1;
    u.cstride = (co + 3) & ~3;
    const size_t cbytes = sizeof(float) * (size_t)u.cstride * dm.S;
    // shared-memory layout: as many blocks per SM as TMEM, shared memory and
    // registers allow, then resident weights, then the deepest weight ring
    u.alias = (dm.Dd + UKC - 1) / UKC == 1;
    const size_t fixed = u.alias ? (size_t)(std::max(u.xchunks, 1) + u.xchunks) * CHUNK_EL
                                 : (size_t)2 * u.xchunks * CHUNK_EL + 2 * CHUNK_EL;
    auto smem_of = [&](int nst) { return sizeof(uint16_t) * (fixed + (size_t)nst * u.np_max * UKC) + cbytes; };
    auto blocks_of = [&](size_t sm) {
        // 228 KB per SM, about 3 KB of static shared memory and 1 KB reserved per block
        return std::min(std::min(512 / u.tcols, reg_blocks), (int)((228 * 1024) / (sm + 4096)));
    };
    int best = -1, best_key = -1;
    for (int nst = 2; nst <= MAX_NST; ++nst) {
        const size_t sm = smem_of(nst);
        if (sm > 200 * 1024) continue;
        const bool res = dm.S == 1 && u.block_chunks == nst;
        const int key = blocks_of(sm) * 16 + (res ? 8 : 0) + nst;
        if (key > best_key) { best_key = key; best = nst; }
    }
    if (best < 0) return false;
    u.nst = best;
    u.resident = dm.S == 1 && u.block_chunks == u.nst;
    u.smem = (int)smem_of(u.nst);
    u.blocks_per_sm = std::max(1, blocks_of(u.smem));
    return true;
}

// blocks of k_mlp_umma that the register file holds at once
int reg_blocks_per_sm() {
    static int blocks = 0;
    if (!blocks) {
        cudaFuncAttributes a;
        if (cudaFuncGetAttributes(&a, k_mlp_umma) == cudaSuccess && a.numRegs > 0)
            blocks = std::max(1, 65536 / (a.numRegs * UTHREADS));
        else
            blocks = 1;
    }
    return blocks;
}

uint16_t bf16_bits(double x) {
    const float f = (float)x;
    uint32_t v;
    std::memcpy(&v, &f, 4);
    if ((v & 0x7f800000u) == 0x7f800000u) return (uint16_t)(v >> 16);
    return (uint16_t)((v + 0x7fffu + ((v >> 16) & 1u)) >> 16);   // round to nearest even
}

}  // namespace

int g_network_kernel = 0;
int network_kernel() { return g_network_kernel; }

bool mlp_umma_supported(const DevModel &dm) {
    UmmaNet u;
    return plan(dm, u);
}

tmd_status mlp_umma_launch(const DevModel &dm, const int32_t *perm, const int32_t *types, int64_t n, const float *G,
                           float *dG, float *e_atom, double *part_e, int *ntile_out, cudaStream_t s) {
    UmmaNet u;
    if (!plan(dm, u)) {
        set_error("network shapes outside the tcgen05 kernel");
        return TMD_ERR_UNIMPLEMENTED;
    }
    static int smem_set = 0;
    if (u.smem > 48 * 1024 && u.smem > smem_set) {
        TMD_CUDA(cudaFuncSetAttribute(k_mlp_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, u.smem));
        smem_set = u.smem;
    }
    const int ntile = (int)((n + UM - 1) / UM);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(ntile, std::max(1, nsm) * u.blocks_per_sm));
    if (ntile > 0)
        TMD_LAUNCH("k_mlp_umma", s, k_mlp_umma<<<grid, UTHREADS, u.smem, s>>>(dm, u, perm, types, n, G, dG, e_atom,
                                                                              part_e, ntile));
    TMD_CUDA(cudaGetLastError());
    *ntile_out = ntile;
    return TMD_OK;
}

// BF16 weights in the operand layout of k_mlp_umma (product order: forward
// layers 0 .. L-1, then backward layers L-1 .. 0); B[n][k] is W_l[n][k]
// forward and W_l[k][n] backward.
tmd_status mlp_umma_build(tmd_model *m, const double *const *weights) {
    DevModel &dm = m->dm;
    const int L = dm.L, S = dm.S;
    if (m->dev_umma) {
        cudaFree(m->dev_umma);
        m->dev_umma = nullptr;
    }
    for (int s = 0; s < TMD_MAX_SPECIES; ++s) dm.ub[s] = nullptr;
    for (int l = 0; l <= L; ++l)
        if (dm.dims[l] % 16) return TMD_OK;   // no BF16 form for these widths
    size_t off = 0;
    int npass[2 * MAX_LAYERS], np[2 * MAX_LAYERS], nk[2 * MAX_LAYERS];
    for (int pr = 0; pr < 2 * L; ++pr) {
        const bool fwd = pr < L;
        const int l = fwd ? pr : 2 * L - 1 - pr;
        const int K = fwd ? dm.dims[l] : dm.dims[l + 1], N = fwd ? dm.dims[l + 1] : dm.dims[l];
        npass[pr] = (N + UNMAX - 1) / UNMAX;
        np[pr] = N / npass[pr];
        nk[pr] = (K + UKC - 1) / UKC;
        if (N % npass[pr] || np[pr] % 16) return TMD_OK;
        dm.uoff[pr] = (int)off;
        off += (size_t)npass[pr] * nk[pr] * np[pr] * UKC;
    }
    const size_t per = (off + 511) & ~size_t(511);   // 1 KiB aligned species blocks
    std::vector<uint16_t> h(per * S, 0);
    for (int s = 0; s < S; ++s) {
        const double *w = weights[s];
        size_t lo[MAX_LAYERS];
        size_t o = 0;
        for (int l = 0; l <= L; ++l) {
            lo[l] = o;
            o += (size_t)dm.dims[l] * dm.dims[l + 1] + dm.dims[l + 1];
        }
        for (int pr = 0; pr < 2 * L; ++pr) {
            const bool fwd = pr < L;
            const int l = fwd ? pr : 2 * L - 1 - pr;
            const int in = dm.dims[l];
            const int K = fwd ? dm.dims[l] : dm.dims[l + 1], N = fwd ? dm.dims[l + 1] : dm.dims[l];
            uint16_t *b = h.data() + per * s + dm.uoff[pr];
            for (int nn = 0; nn < N; ++nn)
                for (int k = 0; k < K; ++k) {
                    const double v = fwd ? w[lo[l] + (size_t)nn * in + k] : w[lo[l] + (size_t)k * in + nn];
                    const int P = nn / np[pr], r = nn % np[pr], c = k / UKC, kk = k % UKC;
                    const size_t idx = ((size_t)P * nk[pr] + c) * np[pr] * UKC + (size_t)(r >> 3) * 512 +
                                       (size_t)(kk >> 3) * 64 + (r & 7) * 8 + (kk & 7);
                    b[idx] = bf16_bits(v);
                }
        }
    }
    void *dev = nullptr;
    cudaError_t e = cudaMalloc(&dev, sizeof(uint16_t) * h.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc tcgen05 weights");
    e = cudaMemcpy(dev, h.data(), sizeof(uint16_t) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dev);
        return cuda_fail(e, "cudaMemcpy tcgen05 weights");
    }
    m->dev_umma = dev;
    for (int s = 0; s < S; ++s) dm.ub[s] = static_cast<const uint16_t *>(dev) + per * s;
    return TMD_OK;
}

tmd_status wait_probe(int32_t *gave_up) {
    int32_t *d = nullptr;
    TMD_CUDA(cudaMalloc(&d, sizeof(int32_t)));
    cudaMemset(d, 0, sizeof(int32_t));
    k_wait_probe<<<1, 32>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int32_t h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
    *gave_up = h;
    return TMD_OK;
}

tmd_status umma_status(int32_t *bits) {
    int32_t v = 0;
    TMD_CUDA(cudaMemcpyFromSymbol(&v, g_umma_status, sizeof(v)));
    const int32_t zero = 0;
    TMD_CUDA(cudaMemcpyToSymbol(g_umma_status, &zero, sizeof(zero)));
    *bits = v;
    return TMD_OK;
}

}  // namespace tmd
