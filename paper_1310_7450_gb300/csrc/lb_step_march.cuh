// lb_step_march.cuh -- the fused lattice-Boltzmann step for wide channels: a TMA-fed row march.
//
// A CTA owns a strip of CW columns (x0 .. x0+CW-1), NC adjacent columns per thread, and marches
// through rows y0..y1-1 of one channel.  The post-collision populations of the previous step stream into a ring of K
// shared-memory slots, one source row per slot: a single 3-D tensor-memory-access copy brings the
// 9 direction planes of that row, columns x0-HP .. x0+CW+HP-1 (HP = 16 bytes of halo on each side,
// so every copy starts on a 16-byte boundary).  The copies run K-2 rows ahead of the arithmetic
// and complete on one mbarrier per slot.
//
// Per row y (one __syncthreads per row):
//   1. moments (Eq. rhoj) of row y+1 for the CW own columns and the two halo columns x0-1, x0+CW,
//      pulled from slots y, y+1, y+2 (Eq. lbupdate, pull form; bounce-back at the walls,
//      Sec. II B); the own populations stay in registers for the next row's collision;
//      the gradient velocity j/R0 goes into a 4-row ring in shared memory;
//   2. barrier; one thread (the last lane) refills the slot of row y with row y+K;
//   3. collision of row y: kappa by three-point differences from the velocity ring, the nlM
//      stress, Sigma^nN, delta rho, n^eq, F_i (Eq. bodyforce), BGK; coalesced stores (with two
//      columns per thread, 8-byte FP32 pairs and 4-byte BF16 pairs).
// The periodic wrap of x is patched into the halo columns of the first and last strip with
// plain loads.  Every mbarrier wait is bounded (MarchCtl::max_wait_ns, 2 s by default): on timeout
// the CTA records LB_ETIMEOUT in the status word, drains its own copies (also bounded) and returns.
#pragma once

#include <cuda.h>

#include "lb_device.cuh"

namespace lbk {

struct MarchItem {
    int x0, y0, y1, pad_;
};

struct MarchCtl {
    const MarchItem* items;
    int n_items;
    int* timeout_flag;  // the channel status word: bit 2 is set when a bounded wait gave up
    long long plane;    // plane stride of the channel's fields (elements)
    long long base;     // plane offset of the channel (its planes start at k * base)
    unsigned long long max_wait_ns;  // limit of every mbarrier wait (0: one non-blocking probe)
    // the last CTA to finish (done_count counts them; zero between launches) stores the channel's
    // status word into status_host (mapped pinned host memory: the host polls it without a copy
    // in the stream) and, on monitor steps (mon set), reduces the item partials into mon[0..3]
    unsigned* done_count = nullptr;
    int* status_host = nullptr;
    double* mon = nullptr;
    long long state_index = 0;
    int with_residual = 0;
};

// A CTA whose wait gave up waits this long for its own copies in flight before it returns.  A
// bulk copy that has not landed after a second means the memory system has failed; the CTA
// leaves then rather than spin without end.
constexpr unsigned long long kMarchDrainNs = 1000000000ull;

// ---- PTX helpers (mbarrier, TMA) ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase with the given parity: mbarrier.try_wait suspends the thread until
// the phase completes or a hardware time limit passes; the loop gives up after max_ns of wall
// time (returns false then).  max_ns = 0: a single non-blocking probe (mbarrier.test_wait).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t max_ns) {
    const uint32_t a = smem_u32(bar);
    if (max_ns == 0) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        return done != 0;
    }
    uint64_t t0 = 0;
    for (uint32_t k = 0;; ++k) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (k == 0) t0 = global_ns();
        else if (global_ns() - t0 > max_ns) return false;
    }
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
// Bulk prefetch of bytes (a multiple of 16, 16-byte aligned) from global memory into L2.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

template <typename T>
struct MarchGeom {
    static constexpr int HP = 16 / (int)sizeof(T);  // halo columns per side (16 bytes)
};

// Shared-memory footprint of the march kernel (bytes).
template <typename T, typename C, int W, int K>
constexpr size_t march_smem_bytes() {
    constexpr int HP = MarchGeom<T>::HP;
    constexpr size_t slot = ((size_t)9 * (W + 2 * HP) * sizeof(T) + 127) / 128 * 128;
    return 128 /*barriers*/ + K * slot + (size_t)4 * (W + 2) * 2 * sizeof(C);
}

// Row loads and stores of NC adjacent values of one plane (8-byte vector accesses for two floats).
template <typename C, int NC>
__device__ __forceinline__ void load_cols(const C* p, C (&v)[NC]) {
    if constexpr (NC == 2 && sizeof(C) == 4) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        v[0] = q.x;
        v[1] = q.y;
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = p[c];
    }
}
template <typename C, int NC>
__device__ __forceinline__ void store_cols(C* p, const C (&v)[NC]) {
    if constexpr (NC == 2 && sizeof(C) == 4) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) p[c] = v[c];
    }
}
// Post-collision populations d + D of NC adjacent nodes (node index of the first in `node`): two
// FP32 values per 8-byte store, two BF16 values (rounded to nearest) per 4-byte store; stochastic
// rounding goes node by node through store_node.
template <typename T, typename C, int NC>
__device__ __forceinline__ void store_cols_pop(T* po, long long P, const C (&d)[NC][9], const C (&D)[NC][9], bool sr,
                                               uint32_t key, uint32_t node) {
    if constexpr (NC == 2 && std::is_same<T, float>::value) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            *reinterpret_cast<float2*>(po + (long long)i * P) = make_float2(d[0][i] + D[0][i], d[1][i] + D[1][i]);
    } else {
        if constexpr (NC == 2 && std::is_same<T, __nv_bfloat16>::value) {
            if (!sr) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    *reinterpret_cast<__nv_bfloat162*>(po + (long long)i * P) =
                        __floats2bfloat162_rn(d[0][i] + D[0][i], d[1][i] + D[1][i]);
                return;
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) store_node<T, C>(po + c, P, d[c], D[c], sr, key, node + (uint32_t)c);
    }
}

// BND = 1: channel ends joined by the generalized periodic boundaries of Sec. II B, and a moving
// Couette wall on the last row (Sec. IV C) if the channel has one; BND = 2: the moving wall only;
// both applied where the populations are pulled (the same rules as the tile kernel's pull9).
// BND = 0: periodic x and bounce-back walls only.
// CW columns per CTA, NC adjacent columns per thread (CW / NC threads).
// Resident CTAs per SM the two-column kernel is compiled for: 7 caps it at 127 registers (no
// spills), 14 warps per SM instead of 10 at its natural 155 (BF16 at 4096 x 4096: 73.8 GLUPS at 7,
// 72.3 at 8, 69.0 at 5; its warps stall mostly on fixed-latency dependencies, which more warps hide).
#ifndef LBK_MARCH_MINB2
#define LBK_MARCH_MINB2 7
#endif
// SCHEME 1: the generalized-Newtonian comparison scheme of Sec. II C (periodic x, bounce-back
// walls, stress mode A), the node's own relaxation rate as in the tile kernel's scheme-1 variant.
// SCHEME 3: the relaxation-time extensions (periodic x, bounce-back walls, either stress mode): the
// node's FP64 fluidity is loaded one row ahead of its use and stored with the step, as in the tile
// kernel's scheme-3 variant (the FP32 kernel then runs 4 CTAs per SM for the registers it needs).
template <typename T, typename C, int SMODE, int CW, int NC, int K, int BND = 0, int SCHEME = 0>
__global__ void __launch_bounds__(CW / NC, NC == 2 ? LBK_MARCH_MINB2 : (SCHEME == 3 ? 4 : 5)) k_step_march(const __grid_constant__ CUtensorMap tmap,
                                                          const StepArgs<T, C> a, const MarchCtl ctl) {
    constexpr int NT = CW / NC;                                      // threads per CTA
    constexpr int HP = MarchGeom<T>::HP;
    constexpr int SW = CW + 2 * HP;                                  // slot row width (elements)
    constexpr size_t SLOT = ((size_t)9 * SW * sizeof(T) + 127) / 128 * 128;
    constexpr uint32_t TX = 9u * SW * sizeof(T);                     // bytes per copy
    constexpr int UW = CW + 2;                                       // velocity ring row width
    static_assert(NT >= 64 && NT % 32 == 0, "the edge patchers and the issuing thread need two warps");

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);               // K mbarriers (<= 16)
    unsigned char* slots = smem + 128;
    C* uring = reinterpret_cast<C*>(slots + K * SLOT);                // [4][UW][2]

    const int t = threadIdx.x;
    const ChanParams<C> P = a.chan[0];
    const int nx = a.nx, ny = P.ny;
    const bool halted = a.status[0] != 0;  // an unstable or timed-out channel takes no more steps

    __shared__ int s_bad;  // set by any thread whose bounded wait gave up; read after a barrier
    __shared__ C s_delta[2];  // BND == 1 with GPBC: rho_out - mean(x = 0), rho_in - mean(x = nx-1)
    // BND == 1 with GPBC: the bracket of the end-crossing rebuild (gpbc_shift_core) of every
    // population that leaves a boundary column across the end, per source row (ring of 8 rows),
    // boundary column c (0: x = 0, directions 3, 6, 7; 1: x = nx-1, directions 1, 5, 8) and
    // direction; six lanes of an edge strip fill one row, the pulls read it
    __shared__ C s_shift[BND == 1 ? 8 : 1][2][3];
    constexpr int TI = NT - 1;  // the thread that issues the copies (last lane; warp 0 computes
                                // the halo columns)
    constexpr int TP = NT - 2;  // the thread that issues the L2 prefetches of residual steps
    if (t == 0) {
        s_bad = 0;
        if (BND == 1 && a.gcol != nullptr) {
            const C* means = a.gcol + 6LL * a.gny;  // [channel][column] means of rho - 1
            s_delta[0] = P.rho_out - means[0];
            s_delta[1] = P.rho_in - means[1];
        }
        prefetch_tmap(&tmap);
        for (int k = 0; k < K; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();

    bool vbad = false;  // some node of this CTA failed the velocity guard (reported when the CTA ends)
    uint32_t nload = 0;  // CTA-uniform count of copies issued (and, in order, consumed)
    bool bad = false;

    auto slot_ptr = [&](uint32_t idx) -> const T* { return reinterpret_cast<const T*>(slots + (idx % K) * SLOT); };
    uint32_t last_issued[K];  // issuing thread: index of the last copy issued into each slot
#pragma unroll
    for (int k = 0; k < K; ++k) last_issued[k] = 0xffffffffu;
    auto issue = [&](uint32_t idx, int x0, int row) {  // issuing thread (TI) only
        uint64_t* b = &bars[idx % K];
        mbar_expect_tx(b, TX);
        tma_load_3d(slots + (idx % K) * SLOT, &tmap, b, x0 - HP, row, 0);
        last_issued[idx % K] = idx;
    };

    for (int item = blockIdx.x; item < ctl.n_items && !bad && !halted; item += gridDim.x) {
        const MarchItem it = ctl.items[item];
        const int x0 = it.x0, y0 = it.y0, y1 = it.y1;
        const int rbase = y0 - 2;                 // first source row of this item
        const int rlast = y1 + 1;                 // last source row
        const uint32_t L0 = nload;                // load index of row rbase
        const bool left_edge = (x0 == 0), right_edge = (x0 + CW == nx);
        const int col0 = NC * t;                  // first own column (relative to x0)
        const int x = x0 + col0;                  // its global column

        // index of the copy holding source row r, and the wait for it
        auto idx_of = [&](int r) -> uint32_t { return L0 + (uint32_t)(r - rbase); };
        auto wait_row = [&](int r) -> bool {
            const uint32_t i = idx_of(r);
            return mbar_wait(&bars[i % K], (i / K) & 1u, ctl.max_wait_ns);
        };
        // periodic wrap: the edge strips' halo columns x0-2, x0-1 (left) or x0+CW, x0+CW+1 (right)
        // come from the other end of the row; threads 0..17 (left) and 32..49 (right) each own
        // one (direction, column) value, loaded two rows before it is patched into its slot
        const bool patcher = (left_edge && t < 18) || (right_edge && t >= 32 && t < 50);
        const int pi = left_edge && t < 18 ? (t >> 1) : ((t - 32) >> 1);             // direction
        const int pc = left_edge && t < 18 ? (nx - 2 + (t & 1)) : ((t - 32) & 1);     // global column
        const int ps = left_edge && t < 18 ? (HP - 2 + (t & 1)) : (HP + CW + ((t - 32) & 1));  // slot column
        auto patch_load = [&](int r) -> T {
            return (r >= 0 && r < ny && r <= rlast) ? a.pin[9 * ctl.base + (long long)pi * ctl.plane + (long long)r * nx + pc] : T(0);
        };
        auto patch_store = [&](int r, T v) {
            if (r >= 0 && r < ny && r <= rlast) const_cast<T*>(slot_ptr(idx_of(r)))[pi * SW + ps] = v;
        };
        // GPBC brackets: lanes 0..5 of the left edge strip's patchers (32..37 on a right edge
        // strip) take one (boundary column, direction) each and evaluate source row r from the
        // slots, which hold the column's raw stored populations (the strip's own edge column, or
        // the halo image of the other end, patched before)
        const bool gpbc_edge = BND == 1 && (left_edge || right_edge) && a.gcol != nullptr;  // CTA-uniform
        const int sl = left_edge ? t : t - 32;
        const bool shifter = gpbc_edge && sl >= 0 && sl < 6;
        auto shift_row = [&](int r) {
            if (r < 0 || r >= ny || r > rlast) return;
            const int c = sl / 3, j = sl - 3 * (sl / 3);
            const int i = c == 1 ? (j == 0 ? 1 : (j == 1 ? 5 : 8)) : (j == 0 ? 3 : (j == 1 ? 6 : 7));
            const int bcol = c == 1 ? (right_edge ? CW - 1 : -1) : (left_edge ? 0 : CW);
            const T* sb = slot_ptr(idx_of(r)) + HP + bcol;
            C e[9], mR, mx, my;
#pragma unroll
            for (int k = 0; k < 9; ++k) e[k] = (C)Store<T>::cvt(sb[k * SW]);
            moments<C>(e, mR, mx, my);
            s_shift[BND == 1 ? (r & 7) : 0][c][j] = gpbc_shift_core<C>(i, mR, mx, my, s_delta[c]);
        };
        // pulled populations of node (col, r) from the slots (col relative to x0, may be -1 or CW):
        // direction i comes from source row r - cy_i, column col - cx_i
        auto pull = [&](int col, int r, C (&d)[9]) {
            const T* s0 = slot_ptr(idx_of(r)) + HP + col;
            if (r > 0 && r < ny - 1) {
                const T* sm = slot_ptr(idx_of(r - 1)) + HP + col;  // source row r-1 (cy = +1)
                const T* sp = slot_ptr(idx_of(r + 1)) + HP + col;  // source row r+1 (cy = -1)
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const T* sr = cy(i) == 1 ? sm : (cy(i) == -1 ? sp : s0);
                    d[i] = (C)Store<T>::cvt(sr[i * SW - cx(i)]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int rs = r - cy(i);
                    if (rs < 0 || rs >= ny) {
                        d[i] = (C)Store<T>::cvt(s0[opp(i) * SW]);  // bounce-back at the wall
                    } else {
                        const T* sr = slot_ptr(idx_of(rs)) + HP + col;
                        d[i] = (C)Store<T>::cvt(sr[i * SW - cx(i)]);
                    }
                }
            }
            if constexpr (BND == 1) {
                if (gpbc_edge) {
                    // the node's true column; the slots hold the raw periodic images, so every
                    // population that crosses an end gets its shift here (Sec. II B):
                    // populations entering x = 0 move with c_x = +1 and leave the column
                    // x = nx-1 (boundary column c = 1); those entering x = nx-1 move with
                    // c_x = -1 and leave x = 0 (c = 0)
                    const int xg = x0 + col;
                    const int X = xg < 0 ? xg + nx : (xg >= nx ? xg - nx : xg);
                    // (direction indices fixed per end: one lane runs this for the whole CTA)
                    if (X == 0) {  // from x = nx-1: directions 1, 5, 8 (source rows r, r-1, r+1)
                        gpbc_add<C>(d[1], 1, s_shift[r & 7][1][0]);
                        if (r > 0) gpbc_add<C>(d[5], 5, s_shift[(r - 1) & 7][1][1]);
                        if (r < ny - 1) gpbc_add<C>(d[8], 8, s_shift[(r + 1) & 7][1][2]);
                    } else if (X == nx - 1) {  // from x = 0: directions 3, 6, 7
                        gpbc_add<C>(d[3], 3, s_shift[r & 7][0][0]);
                        if (r > 0) gpbc_add<C>(d[6], 6, s_shift[(r - 1) & 7][0][1]);
                        if (r < ny - 1) gpbc_add<C>(d[7], 7, s_shift[(r + 1) & 7][0][2]);
                    }
                }
            }
            if constexpr (BND >= 1) {
                if (r == ny - 1 && a.chan[0].moving) zou_he_top<C>(d, a.chan[0].u_wall);
            }
        };
        // the ring holds (u_x, u_y) pairs at even offsets from a 128-byte aligned base: one
        // 8-byte shared access per pair
        using V2 = typename Vec2<C>::type;
        auto put_u = [&](int r, int col, C ux, C uy) {
            V2 v;
            v.x = ux;
            v.y = uy;
            *reinterpret_cast<V2*>(uring + 2 * ((r & 3) * UW + col + 1)) = v;
        };
        auto get_u = [&](const C* p) -> V2 { return *reinterpret_cast<const V2*>(p); };
        auto moments_row = [&](int r, C (&d)[NC][9], C (&dR)[NC], C (&jx)[NC], C (&jy)[NC]) {
            // own columns, then the two halo columns (threads 0 and 1)
            if (r >= 0 && r < ny) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    C ux, uy;
                    pull(col0 + c, r, d[c]);
                    gradient_velocity<C>(d[c], P.gx, dR[c], jx[c], jy[c], ux, uy);
                    put_u(r, col0 + c, ux, uy);
                }
                if (t < 2) {  // the two halo columns, on lanes 0 and 1 of one warp (one pass)
                    const int col = t == 0 ? -1 : CW;
                    C dh[9], hR, hx, hy, ux, uy;
                    pull(col, r, dh);
                    gradient_velocity<C>(dh, P.gx, hR, hx, hy, ux, uy);
                    put_u(r, col, ux, uy);
                }
            }
        };

        // ---- prologue: copies of rows rbase .. rbase+K-1; rows rbase .. rbase+5 waited and patched;
        // moments of rows y0-1, y0 (and of row 2 when the item starts at the bottom wall: the
        // one-sided difference of row 0 needs it)
        if (t == TI) {
            fence_proxy_async();
            for (int r = rbase; r < rbase + K && r <= rlast; ++r) issue(idx_of(r), x0, r);
        }
        nload = L0 + (uint32_t)(rlast - rbase + 1);
        // residual partials (F_RESID / F_MON) of this thread's columns, in the arithmetic type (a
        // few hundred rows at most); the block reduction below runs in double
        C r_du2 = C(0), r_u2 = C(0), r_ux = C(0), r_umax2 = C(0);
        C dcur[NC][9], dnext[NC][9];
        C dRc[NC], jxc[NC], jyc[NC], dRn[NC], jxn[NC], jyn[NC];
        bool ok = true;
        for (int r = rbase; r <= rbase + 5; ++r) ok &= wait_row(r);
        if (!ok) s_bad = 1;
        T pv_a = T(0), pv_b = T(0);
        if (patcher && ok) {  // patch only slots whose copies this thread saw land
            for (int r = rbase; r <= rbase + 5; ++r) patch_store(r, patch_load(r));
            pv_a = patch_load(y0 + 4);
            pv_b = patch_load(y0 + 5);
        }
        __syncthreads();
        if (s_bad) { bad = true; break; }
        if (gpbc_edge) {  // brackets of the rows waited and patched so far (CTA-uniform branch)
            if (shifter)
                for (int r = rbase; r <= rbase + 5; ++r) shift_row(r);
            __syncthreads();
        }
        {
            C dtmp[NC][9], a0[NC], a1[NC], a2[NC];
            moments_row(y0 - 1, dtmp, a0, a1, a2);
            if (y0 == 0) moments_row(2, dtmp, a0, a1, a2);
        }
        moments_row(y0, dcur, dRc, jxc, jyc);
        // the stored flow-induced density, loaded two rows ahead of its use
        const C* drow = a.drho + ctl.base + x;
        C drho_next[NC], drho_next2[NC];
        load_cols<C, NC>(drow + (long long)y0 * nx, drho_next);
        if (y0 + 1 < y1) load_cols<C, NC>(drow + (long long)(y0 + 1) * nx, drho_next2);
        // relaxation-time extensions with a fluidity memory: the node's fluidity (FP64), one row ahead
        const bool fluid = SCHEME == 3 && P.tau_f > C(0);  // CTA-uniform
        const double* phrow = a.phi + ctl.base + x;
        double phi_cur[NC], phi_nxt[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) phi_cur[c] = phi_nxt[c] = 0.0;
        if (fluid)
#pragma unroll
            for (int c = 0; c < NC; ++c) phi_nxt[c] = phrow[(long long)y0 * nx + c];
        // on residual steps the saved velocity of each row is prefetched the same way, and one
        // thread brings the delta rho and saved-velocity rows into L2 four rows before their
        // register loads (a residual step reads 16 B more per node than a plain one, and the
        // two-rows-ahead register pipeline alone covers about one row of DRAM latency)
        const bool resid = (a.flags & F_RESID) != 0;
        const bool mon = (a.flags & (F_RESID | F_MON)) != 0;
        const C* upx = a.uprev + 2 * ctl.base + x;
        const C* upy = upx + ctl.plane;
        auto prefetch_rows = [&](int r) {  // thread TP, residual steps, rows of this item only
            if (r < y1) {
                const long long o = (long long)r * nx + x0;
                prefetch_l2(a.drho + ctl.base + o, CW * sizeof(C));
                prefetch_l2(a.uprev + 2 * ctl.base + o, CW * sizeof(C));
                prefetch_l2(a.uprev + 2 * ctl.base + ctl.plane + o, CW * sizeof(C));
            }
        };
        C upx_next[NC], upy_next[NC], upx_next2[NC], upy_next2[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) upx_next[c] = upy_next[c] = upx_next2[c] = upy_next2[c] = C(0);
        if (resid) {
            if (t == TP)
                for (int r = y0 + 2; r < y0 + 6; ++r) prefetch_rows(r);
            load_cols<C, NC>(upx + (long long)y0 * nx, upx_next);
            load_cols<C, NC>(upy + (long long)y0 * nx, upy_next);
            if (y0 + 1 < y1) {
                load_cols<C, NC>(upx + (long long)(y0 + 1) * nx, upx_next2);
                load_cols<C, NC>(upy + (long long)(y0 + 1) * nx, upy_next2);
            }
        }
        __syncthreads();
        if (t == TI) {
            fence_proxy_async();
            for (int r = rbase + K; r < rbase + K + 2 && r <= rlast; ++r) issue(idx_of(r), x0, r);
        }

        for (int y = y0; y < y1; ++y) {
            // 1. moments of row y+1 (its own populations are the next row's collision input);
            //    edge strips patch row y+4, which the moments of iteration y+2 read first
            if (y + 2 <= rlast && !wait_row(y + 2)) s_bad = 1;
            if (patcher && y + 4 <= rlast) {
                if (!wait_row(y + 4)) s_bad = 1;
                else patch_store(y + 4, pv_a);
                pv_a = pv_b;
                pv_b = patch_load(y + 6);
            }
            moments_row(y + 1, dnext, dRn, jxn, jyn);
            C drho_prev[NC], upx_cur[NC], upy_cur[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                drho_prev[c] = drho_next[c];
                drho_next[c] = drho_next2[c];
                upx_cur[c] = upx_next[c];
                upy_cur[c] = upy_next[c];
            }
            if (y + 2 < y1) load_cols<C, NC>(drow + (long long)(y + 2) * nx, drho_next2);
            if (fluid) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    phi_cur[c] = phi_nxt[c];
                    if (y + 1 < y1) phi_nxt[c] = phrow[(long long)(y + 1) * nx + c];
                }
            }
            if (resid) {
                if (t == TP) prefetch_rows(y + 6);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    upx_next[c] = upx_next2[c];
                    upy_next[c] = upy_next2[c];
                }
                if (y + 2 < y1) {
                    load_cols<C, NC>(upx + (long long)(y + 2) * nx, upx_next2);
                    load_cols<C, NC>(upy + (long long)(y + 2) * nx, upy_next2);
                }
            }
            __syncthreads();
            if (s_bad) { bad = true; break; }
            // 2. refill the slot of row y (no longer read) with row y+K
            if (t == TI && y + K <= rlast) {
                fence_proxy_async();
                issue(idx_of(y + K), x0, y + K);
            }
            // brackets of row y+4: its copy was waited by the shifter lanes (patchers) and its
            // halo patched before the barrier above; the first pull that reads it is that of
            // row y+3, two barriers later
            if (shifter && y + 4 <= rlast) shift_row(y + 4);
            // 3. collision of row y, node by node, then the row's stores
            {
                const long long pn = (long long)y * nx + x;  // first own node
                C so_xx[NC], so_xy[NC], so_yy[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) so_xx[c] = so_xy[c] = so_yy[c] = C(0);
                if (SMODE == 1) {
                    const C* s3 = a.sig3 + 3 * ctl.base + pn;
                    load_cols<C, NC>(s3, so_xx);
                    load_cols<C, NC>(s3 + ctl.plane, so_xy);
                    load_cols<C, NC>(s3 + 2 * ctl.plane, so_yy);
                }
                C D[NC][9], sxx[NC], syy[NC], sxy[NC], drho_new[NC], urx[NC], ury[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int col = col0 + c;
                    const C* uc = uring + 2 * ((y & 3) * UW + col + 1);
                    const V2 ue = get_u(uc + 2), uw = get_u(uc - 2);  // columns col+1, col-1
                    const C ka = C(0.5) * (ue.x - uw.x);
                    const C kc = C(0.5) * (ue.y - uw.y);
                    C kb, ke;
                    const V2 un = get_u(uring + 2 * (((y + 1) & 3) * UW + col + 1));  // row y+1
                    const V2 us = get_u(uring + 2 * (((y + 3) & 3) * UW + col + 1));  // row y-1
                    if (y == 0) {
                        const V2 u0 = get_u(uc);
                        const V2 un2 = get_u(uring + 2 * (((y + 2) & 3) * UW + col + 1));
                        kb = C(0.5) * (C(-3) * u0.x + C(4) * un.x - un2.x);
                        ke = C(0.5) * (C(-3) * u0.y + C(4) * un.y - un2.y);
                    } else if (y == ny - 1) {
                        const V2 u0 = get_u(uc);
                        const V2 us2 = get_u(uring + 2 * (((y + 2) & 3) * UW + col + 1));  // row y-2
                        kb = C(0.5) * (C(3) * u0.x - C(4) * us.x + us2.x);
                        ke = C(0.5) * (C(3) * u0.y - C(4) * us.y + us2.y);
                    } else {
                        kb = C(0.5) * (un.x - us.x);
                        ke = C(0.5) * (un.y - us.y);
                    }
                    NodeState<C> s;
                    C om_n = P.omega;
                    if constexpr (SCHEME == 1) {
                        s = constitutive_gn<C>(P, ka, kb, kc, ke, dRc[c], jxc[c], jyc[c], &om_n);
                    } else if constexpr (SCHEME == 3) {
                        double phi_new;
                        const C tau_M = relaxation_time_ext<C>(P, ka, kb, kc, ke, dRc[c], drho_prev[c], phi_cur[c], &phi_new);
                        s = constitutive<C, SMODE, true>(P, ka, kb, kc, ke, dRc[c], jxc[c], jyc[c], drho_prev[c], so_xx[c],
                                                         so_xy[c], so_yy[c], tau_M);
                        if (fluid) a.phi[ctl.base + pn + c] = phi_new;
                    } else {
                        s = constitutive<C, SMODE>(P, ka, kb, kc, ke, dRc[c], jxc[c], jyc[c], drho_prev[c], so_xx[c],
                                                   so_xy[c], so_yy[c]);
                    }
                    const C rho_h = C(1) + s.dReq - s.drho;
                    vbad |= !velocity_ok<C>(jxc[c], jyc[c], rho_h, a.guard);  // NaN or too fast
                    // the schemes' variants call the collision exactly as the tile kernel's do (the
                    // same expression, so the same contraction into fused multiply-adds)
                    if constexpr (SCHEME == 1) collide_impl<C, true>(P, s, dcur[c], D[c], om_n, C(1) - C(0.5) * om_n, P.gx, C(0));
                    else if constexpr (SCHEME == 3) collide_impl<C, true>(P, s, dcur[c], D[c], P.omega, P.k2, P.gx, C(0));
                    else collide_node<C>(P, s, dcur[c], D[c]);
                    sxx[c] = s.sxx;
                    syy[c] = s.syy;
                    sxy[c] = s.sxy;
                    drho_new[c] = s.drho;
                    urx[c] = ury[c] = C(0);
                    if (a.flags & (F_SAVE_U | F_RESID | F_MON)) {
                        const C ih = Arith<C>::div(C(1), rho_h);
                        urx[c] = jxc[c] * ih;
                        ury[c] = jyc[c] * ih;
                        if (mon) {
                            const C u2 = urx[c] * urx[c] + ury[c] * ury[c];
                            if (resid) {
                                const C dx_ = urx[c] - upx_cur[c], dy_ = ury[c] - upy_cur[c];
                                r_du2 += dx_ * dx_ + dy_ * dy_;
                            }
                            r_u2 += u2;
                            r_ux += urx[c];
                            r_umax2 = fmax(r_umax2, u2);
                        }
                    }
                }
                T* po = a.pout + 9 * ctl.base + pn;
                store_cols_pop<T, C, NC>(po, ctl.plane, dcur, D, (a.flags & F_SR) != 0, a.sr_key, (uint32_t)pn);
                store_cols<C, NC>(a.drho + ctl.base + pn, drho_new);
                if (SMODE == 1) {
                    C* s3 = a.sig3 + 3 * ctl.base + pn;
                    store_cols<C, NC>(s3, sxx);
                    store_cols<C, NC>(s3 + ctl.plane, sxy);
                    store_cols<C, NC>(s3 + 2 * ctl.plane, syy);
                }
                if (a.flags & F_STORE_SIGMA) {  // (the zz plane holds 0 from lb_create on)
                    C* s4 = a.sig4 + 4 * ctl.base + pn;
                    store_cols<C, NC>(s4, sxx);
                    store_cols<C, NC>(s4 + ctl.plane, syy);
                    store_cols<C, NC>(s4 + 3 * ctl.plane, sxy);
                }
                if (a.flags & F_SAVE_U) {
                    C* up_ = a.uprev + 2 * ctl.base + pn;
                    store_cols<C, NC>(up_, urx);
                    store_cols<C, NC>(up_ + ctl.plane, ury);
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) {
#pragma unroll
                for (int i = 0; i < 9; ++i) dcur[c][i] = dnext[c][i];
                dRc[c] = dRn[c];
                jxc[c] = jxn[c];
                jyc[c] = jyn[c];
            }
        }
        __syncthreads();  // every slot read of this item is done before the next item's copies
        if (!bad && mon) {
            // block reduction of (sum du^2, sum u^2, sum u_x, max |u|) into this item's partials
            double v[4] = {(double)r_du2, (double)r_u2, (double)r_ux, (double)r_umax2};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
                v[1] += __shfl_xor_sync(0xffffffffu, v[1], o);
                v[2] += __shfl_xor_sync(0xffffffffu, v[2], o);
                v[3] = fmax(v[3], __shfl_xor_sync(0xffffffffu, v[3], o));
            }
            double* red = reinterpret_cast<double*>(uring);  // the velocity ring is free now
            if ((t & 31) == 0)
                for (int k = 0; k < 4; ++k) red[4 * (t >> 5) + k] = v[k];
            __syncthreads();
            if (t == 0) {
                double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
                for (int w = 0; w < NT / 32; ++w) {
                    s0 += red[4 * w]; s1 += red[4 * w + 1]; s2 += red[4 * w + 2]; s3 = fmax(s3, red[4 * w + 3]);
                }
                double* o = a.partials + 4 * (long long)item;
                o[0] = s0; o[1] = s1; o[2] = s2; o[3] = sqrt(s3);
            }
            __syncthreads();
        }
    }

    if (vbad) atomicOr(a.status, 1);
    if (bad) {
        // record the timeout and drain this CTA's own copies before leaving: a slot is refilled
        // only after every thread's wait on its previous copy succeeded, so the last copy issued
        // into each slot is the only one that can still be in flight (bounded by kMarchDrainNs)
        if (t == TI) {
            atomicOr(ctl.timeout_flag, 2);
            for (int k = 0; k < K; ++k)
                if (last_issued[k] != 0xffffffffu) mbar_wait(&bars[k], (last_issued[k] / K) & 1u, kMarchDrainNs);
        }
        __syncthreads();
    }
    if (ctl.done_count != nullptr) {  // the last CTA to get here: status mirror and monitor
        __shared__ bool s_last;
        __syncthreads();
        if (t == 0) {
            __threadfence();  // this CTA's partials and status bits before its count
            s_last = atomicAdd(ctl.done_count, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_last && t < 32) {
            __threadfence();
            const int st = *(volatile const int*)a.status;
            if (ctl.mon != nullptr)
                monitor_reduce_warp(a.partials, 0, ctl.n_items, st, ctl.mon, nx, ctl.state_index, ctl.with_residual, t);
            if (t == 0) {
                if (ctl.status_host != nullptr) *(volatile int*)ctl.status_host = st;
                *ctl.done_count = 0u;
            }
        }
    }
}

}  // namespace lbk

namespace lbk {
constexpr int kMarchW = 128;  // columns per CTA (one strip)
constexpr int kMarchK = 8;    // shared-memory row slots (copies run K-2 rows ahead)
#ifndef LBK_MARCH_NC_BF16
#define LBK_MARCH_NC_BF16 2
#endif
// Adjacent columns per thread.  BF16 storage moves 56 B per node against FP32's 92, so its step is
// bound by instruction issue: two columns per thread share the per-row address, ring and loop
// work and pack their stores into bf16x2 words (497 -> 366 instructions per node; with 7 CTAs per
// SM 57.7 -> 73.8 GLUPS at 4096 x 4096).  The FP32 step is
// bound by HBM and keeps one column per thread (two measured 4 % slower: a 64-thread CTA at 161
// registers leaves 10 warps per SM to cover the memory latency).  The BF16 boundary variants
// take two columns as well (pressure-driven ends 49.8 -> 59.3, moving wall 55.1 -> 72.0 GLUPS).
template <typename T, int BND>
constexpr int march_nc() { return std::is_same<T, __nv_bfloat16>::value ? LBK_MARCH_NC_BF16 : 1; }

template <typename T, typename C, int SMODE, int BND = 0, int SCHEME = 0>
cudaError_t launch_step_march(const CUtensorMap& map, const StepArgs<T, C>& a, const MarchCtl& ctl, int grid,
                              cudaStream_t s) {
    constexpr int NC = march_nc<T, BND>();
    auto k = k_step_march<T, C, SMODE, kMarchW, NC, kMarchK, BND, SCHEME>;
    const size_t smem = march_smem_bytes<T, C, kMarchW, kMarchK>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    k<<<grid, kMarchW / NC, smem, s>>>(map, a, ctl);
    return cudaGetLastError();
}

template <typename T, typename C, int SMODE, int BND = 0, int SCHEME = 0>
cudaError_t march_occupancy(int* blocks_per_sm) {
    constexpr int NC = march_nc<T, BND>();
    auto k = k_step_march<T, C, SMODE, kMarchW, NC, kMarchK, BND, SCHEME>;
    const size_t smem = march_smem_bytes<T, C, kMarchW, kMarchK>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kMarchW / NC, smem);
}
}  // namespace lbk
