// policy_tc.cuh -- one evaluation of the recurrent policy for every robot, on the tensor cores
// (tcgen05 MMA, accumulators in tensor memory, operands staged by TMA).
//
// The policy (App. A, policy architecture; reading c24):
//   h1 = ReLU(W1 o + b1);  r = sigma(Wi_r h1 + bi_r + Wh_r h + bh_r);  z likewise;
//   n = tanh(Wi_n h1 + bi_n + r (Wh_n h + bh_n));  h' = (1 - z) n + z h;  a = v_max tanh(Wo h' + bo).
// A CTA owns 128 robots (the MMA's M).  Its ten warps:
//   warp 0, lane 0   the TMA producer: K-chunks (64 columns, 128-byte rows, 128-byte swizzle) of
//                    A = [h1 | h] (bf16, this tile's rows) and of the gate weights into a
//                    two-stage ring;
//   warp 1           allocates the tensor memory; its lane 0 issues the MMAs;
//   warps 2-9        two threads per robot (the thread's row = its tensor-memory lane; warps 2-5
//                    take the first half of every block of columns, warps 6-9 the second): the
//                    observation in bf16 for the first product, the zeroed state of robots whose
//                    episode ended, h1 from the first accumulator (bias, ReLU, bf16), then per
//                    block of U hidden units the gates, the new state and the head's partial
//                    sums; the biases and head weights staged once in shared memory.
// Products: D1 [128 x H] = X [128 x 16] W1^T (K = 16, the observation padded); then per unit
// block, four accumulators of U columns: r and z over K = 2H ([h1 | h] against [Wi | Wh]), n_i
// over the first H columns (h1 against Wi_n), n_h over the last H (h against Wh_n).  Operands
// are bf16 (the reading's roundings: o, W1, h1, Wi, Wh and the previous h), accumulation binary32
// in tensor memory; gates, state and head in binary32 (sigma and tanh from the hardware tanh
// approximation, as before).
//
// Every wait on an mbarrier gives up after about two seconds (the kernel then raises a bit in
// the status word, skips its remaining work and still frees its tensor memory).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "env_step.cuh"

namespace rl {
namespace ptc {

constexpr int kM = 128;          // robots per CTA (MMA M)
constexpr int kKc = 64;          // K chunk: 64 bf16 = one 128-byte swizzled row
constexpr int kStages = 2;
constexpr int kHalves = 2;       // epilogue threads per robot (each takes 1 / kHalves of the columns)
constexpr int kEpi = 128 * kHalves;   // epilogue threads
constexpr int kThreads = 64 + kEpi;   // producer warp, MMA warp, epilogue warps
constexpr int kTmemCols = 512;
constexpr int32_t kErrTimeout = kStatusWaitTimeout;  // an mbarrier wait gave up

struct Params {
    const float* obs;           // [rows][od]
    const uint8_t* done_prev;   // [E] episode ended at the previous step, or NULL
    const int32_t* row_env;     // [rows]
    __nv_bfloat16* cat;         // [rows][2H]: h1 (written here), then bf16(h)
    float* h;                   // recurrent state, per tile of 128 robots unit-major:
                                //   h[(tile * H + u) * 128 + robot in tile] (coalesced per unit)
    const __nv_bfloat16* w1;    // [H][16] bf16 (observation columns padded to 16)
    const float* b1;            // [H] bf16-rounded first-layer bias
    const float* bias;          // [4H]: r (bi + bh), z (bi + bh), n_i (bi_n), n_h (bh_n)
    const float* wo;            // [2][H]
    const float* bo;            // [2]
    float* act;                 // [rows][2]
    int32_t* status;
    int rows, od, H, U;
    float vmax;
};

// A resident in shared memory for H <= kResidentH: the whole [128 x 2H] tile, h1 written there
// by the epilogue (no round trip through global memory) and the previous state's chunks fetched
// at the kernel's start; only the weights stream through the ring.  Larger H: A's chunks stream
// through the ring with the weights', h1 through global memory.
constexpr int kResidentH = 256;
__host__ __device__ constexpr bool resident(int H) { return H <= kResidentH; }

// Shared memory (dynamic, 1024-byte aligned): [A (resident case)], the stage ring (per stage:
// [A chunk (streaming case)], gate slots r, z and n (n_i and n_h never share a K-chunk)), X, W1,
// the constants (b1 [H], gate biases [4H], head weights [2H], binary32), the head's partial sums
// [2][128] and the barriers.
__host__ __device__ constexpr size_t a_bytes(int H) { return resident(H) ? (size_t)512 * H : 0; }
__host__ __device__ constexpr size_t stage_a(int H) { return resident(H) ? 0 : 16384; }
__host__ __device__ constexpr size_t stage_bytes(int U, int H) { return stage_a(H) + 3 * (size_t)U * 128; }
__host__ __device__ constexpr size_t x_off(int U, int H) { return a_bytes(H) + kStages * stage_bytes(U, H); }
__host__ __device__ constexpr size_t w1_off(int U, int H) { return x_off(U, H) + 4096; }
__host__ __device__ constexpr size_t c_off(int U, int H) { return w1_off(U, H) + (size_t)H * 32; }
__host__ __device__ constexpr size_t red_off(int U, int H) { return c_off(U, H) + (size_t)7 * H * 4; }
__host__ __device__ constexpr size_t bar_off(int U, int H) { return red_off(U, H) + 2 * 128 * 4; }
__host__ __device__ constexpr size_t smem_bytes(int U, int H) { return bar_off(U, H) + 128 + 1024; }
// the shared-memory slot of gate g (r, z, n_i, n_h) in a stage
__device__ __forceinline__ int gate_slot(int g) { return g < 2 ? g : 2; }

// Index of unit u of robot row_local of tile in the recurrent state.
__device__ __forceinline__ size_t hidx(int tile, int H, int u, int row_local) {
    return ((size_t)tile * H + u) * kM + row_local;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start address, leading- and stride-dimension byte
// offsets (>> 4), the descriptor version bit (46), swizzle mode (bits 61-63: 0 none, 2 128-byte).
__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)swz << 61);
}

// Instruction descriptor of kind::f16: D binary32 (bits 4-5 = 1), A and B bf16 (bits 7-9 and
// 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}"
                 ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity; gives up after ~2 s (status bit, returns false).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int32_t* status) {
    uint32_t ok = 0;
    uint64_t t0 = 0;
    for (int it = 0;; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
        if (it == 0) t0 = now_ns();
        else if ((it & 255) == 0 && now_ns() - t0 > 2000000000ull) {
            atomicOr(status, kErrTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                       uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ float tanh_hw(float v) {
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float sigma_hw(float v) { return fmaf(0.5f, tanh_hw(0.5f * v), 0.5f); }

// Byte offset of element (m, k) in a K-major bf16 tile without swizzle: 8 x 8 core matrices of
// 128 bytes, the two K halves 128 bytes apart (leading-dimension offset), 8-row groups 256
// bytes apart (stride-dimension offset).
__device__ __forceinline__ uint32_t ns_off(int m, int k) {
    return (uint32_t)((m >> 3) * 256 + (k >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2);
}

__global__ void __launch_bounds__(kThreads, 1)
policy_step_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               Params P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the swizzled stages
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int H = P.H, U = P.U;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    const bool res = resident(H);
    unsigned char* as = smem;                        // resident A (H <= kResidentH)
    unsigned char* ring = smem + a_bytes(H);
    unsigned char* xs = smem + x_off(U, H);
    unsigned char* w1s = smem + w1_off(U, H);
    float* cb1 = reinterpret_cast<float*>(smem + c_off(U, H));  // b1 [H]
    float* cbias = cb1 + H;                                       // [4H]
    float* cwo = cbias + 4 * H;                                   // [2H]
    float* red = reinterpret_cast<float*>(smem + red_off(U, H));  // [2][128]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + bar_off(U, H));
    // barriers: full[2], empty[2], d1, h1ready, acc_full, acc_empty, A's previous-state chunks
    // (resident case); then the tmem address
    const uint32_t b_full0 = smem_u32(&bars[0]), b_empty0 = smem_u32(&bars[2]);
    const uint32_t b_d1 = smem_u32(&bars[4]), b_h1 = smem_u32(&bars[5]);
    const uint32_t b_acc = smem_u32(&bars[6]), b_accfree = smem_u32(&bars[7]);
    const uint32_t b_aprev = smem_u32(&bars[8]);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(&bars[9]);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(b_full0 + 8 * s, 1);
            mbar_init(b_empty0 + 8 * s, 1);
        }
        mbar_init(b_d1, 1);
        mbar_init(b_h1, kEpi);
        mbar_init(b_acc, 1);
        mbar_init(b_accfree, kEpi);
        mbar_init(b_aprev, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }

    const int nub = H / U, nk = 2 * H / kKc, kh = H / kKc;
    int row_local = -1, r = -1, half = 0;
    if (warp >= 2) {
        // ---- prologue: this thread's robot (its tensor-memory lane) and its half of the columns
        row_local = 32 * (warp & 3) + lane;
        half = (warp - 2) >> 2;  // 0 .. kHalves - 1
        r = tile * kM + row_local;
        const int et = threadIdx.x - 64;  // 0..255
        const bool valid = r < P.rows;
        // the observation in bf16 (16 columns, zero-padded), K-major without swizzle
#pragma unroll
        for (int kk = 0; kk < 16 / kHalves; ++kk) {
            const int k = (16 / kHalves) * half + kk;
            const float v = (valid && k < P.od) ? P.obs[(size_t)r * P.od + k] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(xs + ns_off(row_local, k)) = __float2bfloat16_rn(v);
        }
        // a robot whose episode ended at the previous step starts from a zero state
        if (valid && P.done_prev && P.done_prev[P.row_env[r]]) {
            const int hc = H / kHalves;
            for (int u = half * hc; u < (half + 1) * hc; ++u) P.h[hidx(tile, H, u, row_local)] = 0.f;
            uint4* cr = reinterpret_cast<uint4*>(P.cat + (size_t)r * 2 * H + H + half * hc);
            for (int q = 0; q < hc / 8; ++q) cr[q] = make_uint4(0u, 0u, 0u, 0u);
        }
        // W1 [H][16] into the same layout, 16-byte pieces (row n, K half q)
        for (int pc = et; pc < 2 * H; pc += kEpi) {
            const int n = pc >> 1, q = pc & 1;
            const uint4 v = *reinterpret_cast<const uint4*>(P.w1 + (size_t)n * 16 + 8 * q);
            *reinterpret_cast<uint4*>(w1s + ns_off(n, 8 * q)) = v;
        }
        // the constants of the epilogues
        for (int q = et; q < H; q += kEpi) cb1[q] = P.b1[q];
        for (int q = et; q < 4 * H; q += kEpi) cbias[q] = P.bias[q];
        for (int q = et; q < 2 * H; q += kEpi) cwo[q] = P.wo[q];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            bool ok = true;
            if (res) {
                // the previous state's chunks of A, at once
                mbar_expect_tx(b_aprev, (uint32_t)(nk - kh) * 16384u);
                for (int kc = kh; kc < nk; ++kc)
                    tma_2d(smem_u32(as + kc * 16384), &tmA, kc * kKc, tile * kM, b_aprev);
            }
            // the weights' chunks go out at once; streamed A chunks wait until h1 is in global
            // memory
            bool h1_ready = res;
            int it = 0;
            for (int ub = 0; ub < nub && ok; ++ub)
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it & 1;
                    const uint32_t ph = (uint32_t)(it >> 1) & 1u;
                    if (!mbar_wait(b_empty0 + 8 * s, ph ^ 1u, P.status)) { ok = false; break; }
                    unsigned char* st = ring + s * stage_bytes(U, H);
                    const bool gi = kc < kh, gh = !gi;  // n_i on h1 columns, n_h on h
                    const uint32_t bytes = (uint32_t)stage_a(H) + 3u * U * 128u;
                    const uint32_t fb = b_full0 + 8 * s;
                    mbar_expect_tx(fb, bytes);
                    for (int g = 0; g < 4; ++g) {
                        if ((g == 2 && !gi) || (g == 3 && !gh)) continue;
                        tma_2d(smem_u32(st + stage_a(H) + gate_slot(g) * U * 128), &tmB, kc * kKc,
                               g * H + ub * U, fb);
                    }
                    if (!res) {
                        if (!h1_ready) {
                            if (!mbar_wait(b_h1, 0, P.status)) { ok = false; break; }
                            h1_ready = true;
                        }
                        tma_2d(smem_u32(st), &tmA, kc * kKc, tile * kM, fb);
                    }
                }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: D1, then the gate accumulators of each unit block
        if (lane == 0) {
            for (int n0 = 0; n0 < H; n0 += 256) {
                const int N = (H - n0) < 256 ? (H - n0) : 256;
                mma_bf16(tmem + n0, mdesc(smem_u32(xs), 128, 256, 0),
                         mdesc(smem_u32(w1s + (n0 / 8) * 256), 128, 256, 0), idesc_bf16(kM, N), 0u);
            }
            mma_commit(b_d1);
            // the accumulators reuse D1's columns once h1 has been read out
            bool ok = mbar_wait(b_h1, 0, P.status);
            if (res) ok = mbar_wait(b_aprev, 0, P.status) && ok;
            tc_fence_after();
            const uint32_t idesc = idesc_bf16(kM, U);
            int it = 0;
            for (int ub = 0; ub < nub && ok; ++ub) {
                if (ub > 0) {
                    ok = mbar_wait(b_accfree, (uint32_t)(ub - 1) & 1u, P.status);
                    tc_fence_after();
                    if (!ok) break;
                }
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it & 1;
                    const uint32_t ph = (uint32_t)(it >> 1) & 1u;
                    if (!mbar_wait(b_full0 + 8 * s, ph, P.status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t st = smem_u32(ring + s * stage_bytes(U, H));
                    const uint32_t sa = res ? smem_u32(as + kc * 16384) : st;
                    const bool gi = kc < kh, gh = !gi;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        if ((g == 2 && !gi) || (g == 3 && !gh)) continue;
                        const bool first = (g == 3) ? (kc == kh) : (kc == 0);
                        const uint32_t sb = st + (uint32_t)stage_a(H) + gate_slot(g) * U * 128;
#pragma unroll
                        for (int ks = 0; ks < kKc / 16; ++ks)
                            mma_bf16(tmem + g * U, mdesc(sa + ks * 32, 16, 1024, 2),
                                     mdesc(sb + ks * 32, 16, 1024, 2), idesc,
                                     (first && ks == 0) ? 0u : 1u);
                    }
                    mma_commit(b_empty0 + 8 * s);  // the stage is free once these MMAs are done
                }
                mma_commit(b_acc);
            }
        }
    } else {
        // ---- epilogues, two threads per robot (halves of the columns)
        const bool valid = r < P.rows;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        bool ok = mbar_wait(b_d1, 0, P.status);
        tc_fence_after();
        // h1 = ReLU(D1 + b1) in bf16 into the first H columns of the row of A
        for (int c0 = half * (H / kHalves); c0 < (half + 1) * (H / kHalves); c0 += 32) {
            float v[32];
            tmem_ld32(lane_base + c0, v);
            tmem_wait_ld();
            {
                uint4* dst = reinterpret_cast<uint4*>(P.cat + (size_t)r * 2 * H + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 ba = *reinterpret_cast<const float4*>(cb1 + c0 + 8 * q);
                    const float4 bb = *reinterpret_cast<const float4*>(cb1 + c0 + 8 * q + 4);
                    const float bq[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
                    __nv_bfloat162 pk[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        pk[j] = __floats2bfloat162_rn(fmaxf(v[8 * q + 2 * j] + bq[2 * j], 0.f),
                                                      fmaxf(v[8 * q + 2 * j + 1] + bq[2 * j + 1], 0.f));
                    if (res) {
                        // into resident A, 128-byte swizzle: 16-byte unit j of row m at
                        // m * 128 + ((j ^ (m & 7)) << 4) within its 64-column chunk
                        const int c = c0 + 8 * q, j = (c & 63) >> 3;
                        *reinterpret_cast<uint4*>(as + (c >> 6) * 16384 + row_local * 128 +
                                                  ((j ^ (row_local & 7)) << 4)) =
                            *reinterpret_cast<uint4*>(pk);
                    } else if (valid) {
                        dst[q] = *reinterpret_cast<uint4*>(pk);
                    }
                }
            }
        }
        if (res) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        else asm volatile("fence.proxy.async.global;" ::: "memory");
        tc_fence_before();
        mbar_arrive(b_h1);
        float a0 = 0.f, a1 = 0.f;
        // slices of 16 units: spu per unit block for this thread's half of the columns; the
        // state of the next slice is loaded while the current one is computed (the first one
        // while the products run)
        const int spu = U / kHalves / 16, ns = nub * spu;
        auto slice_u0 = [&](int si) { return (si / spu) * U + half * (U / kHalves) + (si % spu) * 16; };
        float hnext[16];
        if (valid) {
#pragma unroll
            for (int j = 0; j < 16; ++j) hnext[j] = P.h[hidx(tile, H, slice_u0(0) + j, row_local)];
        }
        for (int si = 0; si < ns; ++si) {
            const int ub = si / spu;
            if (si % spu == 0) {
                ok = mbar_wait(b_acc, (uint32_t)ub & 1u, P.status) && ok;
                tc_fence_after();
            }
            const int u0 = slice_u0(si), c0 = u0 - ub * U;
            float vr[16], vz[16], vi[16], vh[16];
            tmem_ld16(lane_base + 0 * U + c0, vr);
            tmem_ld16(lane_base + 1 * U + c0, vz);
            tmem_ld16(lane_base + 2 * U + c0, vi);
            tmem_ld16(lane_base + 3 * U + c0, vh);
            float hv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) hv[j] = hnext[j];
            if (valid && si + 1 < ns) {
                const int un = slice_u0(si + 1);
#pragma unroll
                for (int j = 0; j < 16; ++j) hnext[j] = P.h[hidx(tile, H, un + j, row_local)];
            }
            tmem_wait_ld();
            if (valid) {
                float hb[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int u = u0 + 4 * q;
                    const float4 br = *reinterpret_cast<const float4*>(cbias + u);
                    const float4 bz = *reinterpret_cast<const float4*>(cbias + H + u);
                    const float4 bi = *reinterpret_cast<const float4*>(cbias + 2 * H + u);
                    const float4 bh = *reinterpret_cast<const float4*>(cbias + 3 * H + u);
                    const float4 w0 = *reinterpret_cast<const float4*>(cwo + u);
                    const float4 w1v = *reinterpret_cast<const float4*>(cwo + H + u);
                    const float brv[4] = {br.x, br.y, br.z, br.w}, bzv[4] = {bz.x, bz.y, bz.z, bz.w};
                    const float biv[4] = {bi.x, bi.y, bi.z, bi.w}, bhv[4] = {bh.x, bh.y, bh.z, bh.w};
                    const float w0v[4] = {w0.x, w0.y, w0.z, w0.w}, w1w[4] = {w1v.x, w1v.y, w1v.z, w1v.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int c = 4 * q + j;
                        const float rg = sigma_hw(vr[c] + brv[j]);
                        const float zg = sigma_hw(vz[c] + bzv[j]);
                        const float ng = tanh_hw(vi[c] + biv[j] + rg * (vh[c] + bhv[j]));
                        const float hn = (1.f - zg) * ng + zg * hv[c];
                        hb[c] = hn;
                        a0 += w0v[j] * hn;
                        a1 += w1w[j] * hn;
                    }
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) P.h[hidx(tile, H, u0 + j, row_local)] = hb[j];
                if (res || nub == 1) {
                    // nothing reads the h half of A in global memory any more (resident A was
                    // fetched before the first product; or every product has completed): the
                    // new state in bf16 straight into it for the next step
                    uint4* cd = reinterpret_cast<uint4*>(P.cat + (size_t)r * 2 * H + H + u0);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        __nv_bfloat162 pk[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            pk[j] = __floats2bfloat162_rn(hb[8 * q + 2 * j], hb[8 * q + 2 * j + 1]);
                        cd[q] = *reinterpret_cast<uint4*>(pk);
                    }
                }
            }
            if (si % spu == spu - 1) {
                tc_fence_before();
                mbar_arrive(b_accfree);
            }
        }
        // the head: the second half's partial sums through shared memory
        if (kHalves == 2) {
            if (half == 1) {
                red[row_local] = a0;
                red[128 + row_local] = a1;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kEpi) : "memory");
            if (half == 0) {
                a0 += red[row_local];
                a1 += red[128 + row_local];
            }
        }
        if (half == 0 && valid) {
            P.act[2 * (size_t)r] = P.vmax * tanhf(a0 + P.bo[0]);
            P.act[2 * (size_t)r + 1] = P.vmax * tanhf(a1 + P.bo[1]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // with several unit blocks, once every product of this CTA has completed (the last
    // accumulator was read): the new state in bf16 into the h half of A for the next step
    if (!res && nub > 1 && warp >= 2 && r < P.rows) {
        const int hc = H / kHalves;
        uint2* cd = reinterpret_cast<uint2*>(P.cat + (size_t)r * 2 * H + H + half * hc);
        for (int q = 0; q < hc / 4; ++q) {
            const int u = half * hc + 4 * q;
            const float4 v = make_float4(P.h[hidx(tile, H, u, row_local)], P.h[hidx(tile, H, u + 1, row_local)],
                                         P.h[hidx(tile, H, u + 2, row_local)], P.h[hidx(tile, H, u + 3, row_local)]);
            __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t*>(&lo);
            pk.y = *reinterpret_cast<uint32_t*>(&hi);
            cd[q] = pk;
        }
    }
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols) : "memory");
    }
}

}  // namespace ptc
}  // namespace rl
