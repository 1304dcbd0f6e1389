// k_tc.cu -- tensor-core projection O = (X - c) W^T on sm_103a (Sec. 3.1
// Eq. rotate with the combined PCA + segment-rotation matrix of Sec. 5.1).
//
// One CTA computes a 128-row x NP-column tile of O (NP <= 256, a multiple of
// 16 chosen per model so that the column passes are balanced) over K = d:
//   warp 0      TMA producer: the FP32 X tile (128 rows x 32 values per box,
//               128-byte swizzle, staged) and the W operand tile(s).  W is a
//               model constant, stored in global memory already cut into
//               the (pass, K block) tiles of the shared-memory layout the
//               MMA reads (NP rows of 64 bytes, 64-byte swizzle), so each
//               operand tile is one contiguous bulk copy instead of NP
//               64-byte rows of a tensor copy;
//   warp 1      TMEM owner and MMA issuer: the whole warp runs the K loop
//               and one lane, elected inside each instruction, issues the
//               tcgen05.mma and commits (a loop run by one lane alone issued
//               them about 4% slower at d = 960, FP32); accumulator 128
//               lanes x NP FP32 columns in TMEM;
//   warps 2-9   converters, then epilogue.  Two groups of four warps take
//               alternate K blocks (two blocks in conversion at once); in a
//               group one thread per tile row reads the staged X values,
//               centres and scales them with one FMA against -c*s kept in
//               shared memory, converts them into the A operand(s) and
//               accumulates |x - c|^2; after the K loop each warp drains its
//               TMEM lane quadrant for alternate 32-column blocks with
//               tcgen05.ld.  Every form writes each row's A values to TMEM
//               with tcgen05.st (16-column buffers per stage beside the
//               accumulators: one for BF16 / FP8, a hi and a lo buffer for
//               the split) and the MMAs read A from there, which takes the A
//               tiles' writes and their reads by the MMAs off the shared
//               memory ports: the split form was bound by shared-memory
//               bandwidth (per K block the TMA, the converters and the MMAs
//               moved 147 KB through it, 1,150 cycles at 128 B per clock).
// Operand rows are 64 bytes per stage (32 FP16/BF16 or 64 E4M3 values), so
// three or more stages fit in shared memory.
// Precision modes:
//   kSplit  FP32: A = a_hi + a_lo and B = b_hi + b_lo as FP16 pairs (scaled by
//           powers of two), D = a_hi b_hi + (a_hi b_lo + a_lo b_hi) with FP32
//           accumulation.  The tensor core's accumulation is not rounded to
//           nearest: each MMA shrinks the accumulator by a fraction of an
//           FP32 ulp, which over K = 3072 in one accumulator (576 MMAs) came
//           to a 1e-5 loss of |o|.  The two correction products therefore go
//           to a second accumulator (TMEM columns 256..511, 2^-11 of the
//           main term, so its own loss does not count), the main one takes
//           a third of the MMAs, and the epilogue adds the two in FP32;
//   kBF16   one BF16 product;
//   kFP8    one E4M3 product (kind::f8f6f4), per-segment scales on W.
// All waits are bounded (about 2 s); a timed-out wait raises an error flag,
// every role leaves its loop, in-flight copies and MMAs are drained, TMEM is
// freed and the kernel returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "saq_internal.h"

namespace saq {

namespace {

enum Mode { kSplit = 0, kBF16 = 1, kFP8 = 2 };

constexpr int kBM = 128;            // rows per tile (UMMA M)
constexpr int kNPMax = 256;         // output columns per tile at most (UMMA N)
// the split form's column passes: two accumulators of at most 192 columns
// and four hi/lo A buffers of 32 columns share the 512 TMEM columns
constexpr int kSplitNP = 192;
// X boxes are prefetched into L2 this many K blocks ahead (measured at d =
// 960 / 1536 / 3072: 4 ahead beats 8 by 1% / 0.2% / 2-4% and 16 or 32 lose
// 1-13%; without a prefetch the projection is 8-20% slower)
constexpr int kPrefetch = 4;
constexpr int kAcc2 = 256;          // TMEM column of the split mode's correction accumulator
constexpr int kConvWarps = 8;
// error word: 1..5 the role whose wait timed out; kErrRange an input row
// outside the operand format's range (or not finite)
constexpr int kErrRange = 16;
constexpr int kThreads = 64 + 32 * kConvWarps;
// The double-buffered persistent form (BF16, FP8): four more warps that only
// drain accumulators, so that one tile's epilogue runs beside the next
// tile's MMAs.
constexpr int kEpiWarps = 4;
constexpr int kThreadsDb = kThreads + 32 * kEpiWarps;
constexpr uint32_t kXBox = 16384;   // 128 rows x 128 bytes of staged FP32
constexpr uint32_t kBTile = 16384;  // 256 rows x 64 bytes

// Per stage: XBOX staged X boxes and NB W-operand tiles in shared memory (the
// A operand of the stage lives in TMEM).
template <int MODE> struct Cfg;
template <> struct Cfg<kSplit> {  // 32 FP16 per row per stage, A hi/lo in TMEM
    static constexpr int BK = 32, STAGES = 4, NB = 2, XBOX = 1, TMEM = 512;
};
template <> struct Cfg<kBF16> {  // 32 BF16 per row per stage, A in TMEM
    static constexpr int BK = 32, STAGES = 6, NB = 1, XBOX = 1, TMEM = 512;
};
template <> struct Cfg<kFP8> {  // 64 E4M3 per row per stage, A in TMEM
    static constexpr int BK = 64, STAGES = 4, NB = 1, XBOX = 2, TMEM = 512;
};
// TMEM column of the A buffers (16 columns, 64 bytes of a row, each):
// BF16 / FP8 one per stage after the accumulator (columns 256 ..); the split
// form a hi (part 0) and a lo (part 1) buffer per stage in the gaps beside
// its accumulators (main 0 .. 191, correction 256 .. 447): stages 0-1 at
// 192 .., stages 2-3 at 448 ..
constexpr uint32_t kTA = 256;
static_assert(kTA + 16u * Cfg<kBF16>::STAGES <= 512u && kTA + 16u * Cfg<kFP8>::STAGES <= 512u,
              "A buffers exceed the TMEM allocation");
static_assert(Cfg<kSplit>::STAGES == 4 && kSplitNP <= 192 && kAcc2 == 256 &&
                  kAcc2 + kSplitNP <= 448,
              "split-form TMEM map: accumulators and A buffers overlap");
// The double-buffered BF16 / FP8 form: accumulators at columns 0 and kAccDb
// (column passes of at most kAccDb), the A buffers (six or four) from kTADb.
constexpr uint32_t kAccDb = 208, kTADb = 416;
static_assert(2u * kAccDb <= kTADb && kTADb + 16u * Cfg<kBF16>::STAGES <= 512u &&
                  kTADb + 16u * Cfg<kFP8>::STAGES <= 512u,
              "double-buffered TMEM map: accumulators and A buffers overlap");
template <int MODE> __host__ __device__ constexpr uint32_t ta_col(int s, int part) {
    return MODE == kSplit ? (s < 2 ? 192u + 32u * (uint32_t)s : 448u + 32u * (uint32_t)(s - 2)) +
                                16u * (uint32_t)part
                          : kTA + 16u * (uint32_t)s;
}

template <int MODE> constexpr uint32_t stage_bytes() {
    return (uint32_t)Cfg<MODE>::XBOX * kXBox + (uint32_t)Cfg<MODE>::NB * kBTile;
}
template <int MODE> constexpr uint32_t b_offset() { return (uint32_t)Cfg<MODE>::XBOX * kXBox; }
// A CTA that allocates all 512 TMEM columns must be alone on its SM (an
// allocation beyond the free columns waits for a co-resident CTA to free
// its own): its stages alone take more than half of the 228 KB of an SM.
static_assert(Cfg<kSplit>::STAGES * stage_bytes<kSplit>() > 228u * 1024u / 2u &&
                  Cfg<kBF16>::STAGES * stage_bytes<kBF16>() > 228u * 1024u / 2u &&
                  Cfg<kFP8>::STAGES * stage_bytes<kFP8>() > 228u * 1024u / 2u,
              "two CTAs per SM would share 512 TMEM columns");
// barriers (full, conv, empty per stage; the accumulators' full (up to two);
// for the persistent kernels the tile ring's full and empty (up to four
// slots each), the accumulators' empty (up to two) and the final MMA
// barrier, then the ring's entries), the TMEM address and the abort flag,
// ahead of the row-norm halves
constexpr uint32_t kBarArea = 512;
template <int MODE> constexpr uint32_t bar_bytes() {
    return 3u * 8u * Cfg<MODE>::STAGES + 2u * 8u + 8u * 8u + 2u * 8u + 8u + 4u * 8u + 8u;
}
static_assert(bar_bytes<kSplit>() <= kBarArea && bar_bytes<kBF16>() <= kBarArea &&
                  bar_bytes<kFP8>() <= kBarArea,
              "barriers overflow their shared-memory area");
// dynamic shared memory: stages, barriers, the row-norm halves, -c*s
template <int MODE> constexpr uint32_t smem_bytes(int dpad) {
    return Cfg<MODE>::STAGES * stage_bytes<MODE>() + 1024 + kBarArea + 512 + 4u * (uint32_t)dpad;
}
// every form fits the 227 KB a CTA may opt into at the largest supported d (6144)
static_assert(smem_bytes<kSplit>(6144) <= 227u * 1024u && smem_bytes<kBF16>(6144) <= 227u * 1024u &&
                  smem_bytes<kFP8>(6144) <= 227u * 1024u,
              "stages exceed the dynamic shared memory of one CTA");

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bound of the drain waits (in-flight copies and MMAs at exit), which always
// end; the role waits of the pipeline take their bound from the launch
// (kWaitNs unless saq_set_wait_limit changed it).
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s
// Bounded wait for the phase of `parity` to complete.  Returns false on a
// timeout after `limit_ns` (after raising the flags) or when another role
// already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int *err, int code, uint64_t limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    // a bound below 10 us is checked on every poll, so that a wait longer
    // than it gives up however few polls it took
    const uint32_t every = limit_ns < 10000ull ? 0u : 255u;
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & every) == 0u) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > limit_ns) {
                *abort_flag = 1;
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}
// mbar_wait by every lane of a converged warp; the result is the same in all
// of them.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int *err, int code, uint64_t limit_ns) {
    const bool r = mbar_wait(bar, parity, abort_flag, err, code, limit_ns);
    return __all_sync(0xffffffffu, r);
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// pull a box of the tensor into L2 ahead of its load (no shared memory)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     (uint64_t)map),
                 "r"(x), "r"(y)
                 : "memory");
}
// contiguous global -> shared copy (16-byte aligned, a multiple of 16 bytes)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// K-major operand, 64-byte rows with the 64-byte swizzle, 8-row groups 512
// bytes apart.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;           // leading byte offset (unused for this layout)
    d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;           // descriptor version
    d |= (uint64_t)4 << 61;           // 64-byte swizzle
    return d;
}
template <int MODE> __host__ __device__ constexpr uint32_t umma_idesc_base() {
    uint32_t d = 1u << 4;                           // accumulate in FP32
    if (MODE == kBF16) d |= (1u << 7) | (1u << 10);  // A, B = BF16 (F16 and E4M3 encode as 0)
    d |= (uint32_t)(kBM >> 4) << 24;
    return d;
}
// 16 consecutive 32-bit TMEM columns of the warp's lane quadrant, one word per
// column from each thread (its own lane), and the wait for them
__device__ __forceinline__ void tmem_st16(uint32_t ta, const uint32_t (&w)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(ta),
        "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]),
        "r"(w[8]), "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// tcgen05.mma with the A operand in TMEM (column address `atm`, 128 lanes),
// B from shared memory (descriptor b), D in TMEM at dtm, and tcgen05.commit
// of the MMAs issued so far to an mbarrier.  Both are executed by a whole,
// converged warp, and one lane, elected inside the instruction sequence,
// issues them: a loop run by the whole warp keeps its control flow and the
// instructions' operands warp-uniform, which the MMA issue rate depends on.
template <int MODE>
__device__ __forceinline__ void umma_ta_elect(uint32_t dtm, uint32_t atm, uint64_t b, uint32_t idesc,
                                              uint32_t acc) {
    if (MODE == kFP8) {
        asm volatile(
            "{\n .reg .pred e, p;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " @e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtm),
            "r"(atm), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred e, p;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
            " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtm),
            "r"(atm), "l"(b), "r"(idesc), "r"(acc));
    }
}
__device__ __forceinline__ void umma_commit_elect(uint64_t *bar) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
            smem_u32(bar))
        : "memory");
}
// 32 consecutive accumulator columns of the warp's lane quadrant (one wait)
__device__ __forceinline__ void tmem_ld32(uint32_t ta, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// the same 32 columns of both accumulators of the split mode, one wait
__device__ __forceinline__ void tmem_ld32x2(uint32_t ta, uint32_t tb, float (&v)[32],
                                            float (&w)[32]) {
    uint32_t r[32], q[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%64];\n"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%65];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]), "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15]), "=r"(q[16]), "=r"(q[17]), "=r"(q[18]), "=r"(q[19]), "=r"(q[20]), "=r"(q[21]), "=r"(q[22]), "=r"(q[23]), "=r"(q[24]), "=r"(q[25]), "=r"(q[26]), "=r"(q[27]), "=r"(q[28]), "=r"(q[29]), "=r"(q[30]), "=r"(q[31])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        v[i] = __uint_as_float(r[i]);
        w[i] = __uint_as_float(q[i]);
    }
}
__device__ __forceinline__ void named_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ uint32_t pack_h2(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }
__device__ __forceinline__ uint32_t pack_b2(__nv_bfloat162 h) {
    return *reinterpret_cast<uint32_t *>(&h);
}

// 16-byte chunk `c` of row `r` of a staged FP32 box (128-byte rows, 128-byte
// swizzle).
__device__ __forceinline__ uint32_t swz128(int r, int c) {
    return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

// One K block of one tile row: the row's staged X values (stage st, row r)
// centred and scaled with one FMA against -c * s (mk), converted into the A
// operand words (split: hi in wa, lo in wl), and their squares added to nrm.
template <int MODE>
__device__ __forceinline__ void convert_block(const uint8_t *st, const float *mk, int r,
                                              float x_scale, float &nrm, uint32_t (&wa)[16],
                                              uint32_t (&wl)[16]) {
    if (MODE == kFP8) {
        // 4 chunks of 16 E4M3 (64 values) per thread, from the two staged boxes
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int ac = i;  // operand chunk: values ac*16 .. ac*16+15
            const uint8_t *xb = st + (i >> 1) * kXBox;
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = (i & 1) * 4 + e;  // staged chunk within its box
                const float4 x = *reinterpret_cast<const float4 *>(xb + swz128(r, c));
                const float4 m = *reinterpret_cast<const float4 *>(mk + ac * 16 + e * 4);
                const float y0 = fmaf(x.x, x_scale, m.x), y1 = fmaf(x.y, x_scale, m.y);
                const float y2 = fmaf(x.z, x_scale, m.z), y3 = fmaf(x.w, x_scale, m.w);
                nrm = fmaf(y0, y0, nrm); nrm = fmaf(y1, y1, nrm);
                nrm = fmaf(y2, y2, nrm); nrm = fmaf(y3, y3, nrm);
                const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(
                    make_float2(y0, y1), __NV_SATFINITE, __NV_E4M3);
                const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
                    make_float2(y2, y3), __NV_SATFINITE, __NV_E4M3);
                w[e] = (uint32_t)lo | ((uint32_t)hi << 16);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) wa[4 * i + e] = w[e];  // values 16i + 4e .. + 3
        }
    } else {
        // 4 chunks of 8 values (32 values) per thread from the staged box
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int ac = i;  // operand chunk: values ac*8 .. ac*8+7
            const float4 x0 = *reinterpret_cast<const float4 *>(st + swz128(r, 2 * ac));
            const float4 x1 = *reinterpret_cast<const float4 *>(st + swz128(r, 2 * ac + 1));
            const float4 m0 = *reinterpret_cast<const float4 *>(mk + ac * 8);
            const float4 m1 = *reinterpret_cast<const float4 *>(mk + ac * 8 + 4);
            float y[8] = {fmaf(x0.x, x_scale, m0.x), fmaf(x0.y, x_scale, m0.y),
                          fmaf(x0.z, x_scale, m0.z), fmaf(x0.w, x_scale, m0.w),
                          fmaf(x1.x, x_scale, m1.x), fmaf(x1.y, x_scale, m1.y),
                          fmaf(x1.z, x_scale, m1.z), fmaf(x1.w, x_scale, m1.w)};
#pragma unroll
            for (int e = 0; e < 8; ++e) nrm = fmaf(y[e], y[e], nrm);
            if (MODE == kBF16) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    w[e] = pack_b2(__floats2bfloat162_rn(y[2 * e], y[2 * e + 1]));
#pragma unroll
                for (int e = 0; e < 4; ++e) wa[4 * i + e] = w[e];  // values 8i + 2e, + 1
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {  // values 8i + 2e, + 1
                    const __half2 hh = __floats2half2_rn(y[2 * e], y[2 * e + 1]);
                    const float2 hf = __half22float2(hh);
                    wa[4 * i + e] = pack_h2(hh);
                    wl[4 * i + e] =
                        pack_h2(__floats2half2_rn(y[2 * e] - hf.x, y[2 * e + 1] - hf.y));
                }
            }
        }
    }
}

// The epilogue of one tile row (thread of row r in lane quadrant tq, column
// blocks first, first + step, ... of 32): accumulator columns scaled per output column
// into O (row-major with stride ldo, or interleaved by groups of 32 rows when
// il), and with vmax != NULL the running max |o| of each kept segment.
template <int MODE>
__device__ __forceinline__ void tile_epilogue(uint32_t tq, int first, int step, int lane, int r,
                                              int64_t row0,
                                              bool row_ok, int np, int col0, int dk,
                                              const float *__restrict__ col_scale,
                                              float *__restrict__ O, int64_t ldo, int il,
                                              float *__restrict__ vmax, const SegCols &segc) {
    float *orow = O + (row0 + r) * ldo;
    // interleaved: column `col` of row R at ((R / 32) * dk + col) * 32 + R % 32
    float *ogrp = O + (((row0 + r) >> 5) * (int64_t)dk << 5) + lane;
    // running max |o| of the current kept segment (interleaved layout only)
    const bool want_vmax = il && vmax != nullptr;
    float *vgrp = want_vmax ? vmax + (((row0 + r) >> 5) * (int64_t)segc.nk << 5) + lane
                            : nullptr;
    int si = 0;
    float mx = 0.f;
    // 32-column blocks, alternating between the two threads of a row; a
    // block past np reads accumulator columns the allocation holds
    // (np <= 256) and scales from the padded scale vector
#pragma unroll 1
    for (int b = first; b < ((np + 31) >> 5); b += step) {
        const int c = b << 5;
        const int cb = col0 + c;  // first output column of the block
        float4 sc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) sc[i] = __ldg(reinterpret_cast<const float4 *>(col_scale + cb) + i);
        float v[32];
        if (MODE == kSplit) {
            float v2[32];
            tmem_ld32x2(tq + (uint32_t)c, tq + (uint32_t)(kAcc2 + c), v, v2);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += v2[i];
        } else {
            tmem_ld32(tq + (uint32_t)c, v);
        }
        if (!row_ok || cb >= dk) continue;
        const int cn = min(min(32, np - c), dk - cb);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            v[4 * i] *= sc[i].x; v[4 * i + 1] *= sc[i].y;
            v[4 * i + 2] *= sc[i].z; v[4 * i + 3] *= sc[i].w;
        }
        if (cn == 32) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (il) ogrp[(int64_t)(cb + i) << 5] = v[i];
                else orow[cb + i] = v[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (i >= cn) break;
                if (il) ogrp[(int64_t)(cb + i) << 5] = v[i];
                else orow[cb + i] = v[i];
            }
        }
        if (want_vmax) {
            while (cb >= segc.end[si]) {
                if (mx > 0.f) atomicMax((int *)(vgrp + ((int64_t)si << 5)), __float_as_int(mx));
                mx = 0.f;
                ++si;
            }
            if (cb + cn <= segc.end[si]) {  // the block lies in one segment
#pragma unroll
                for (int i = 0; i < 32; ++i) mx = fmaxf(mx, i < cn ? fabsf(v[i]) : 0.f);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    if (i >= cn) break;
                    while (cb + i >= segc.end[si]) {
                        if (mx > 0.f)
                            atomicMax((int *)(vgrp + ((int64_t)si << 5)), __float_as_int(mx));
                        mx = 0.f;
                        ++si;
                    }
                    mx = fmaxf(mx, fabsf(v[i]));
                }
            }
        }
    }
    if (want_vmax && row_ok && mx > 0.f)
        atomicMax((int *)(vgrp + ((int64_t)si << 5)), __float_as_int(mx));
}

// The work of one CTA: row tile `tile`, column pass `pass` of one model
// (tmx: the tensor map of its X rows, in parameter space).
template <int MODE>
__device__ __forceinline__ void proj_tile(
    const CUtensorMap *tmxp, int64_t tile, int pass, const uint8_t *__restrict__ wt0,
    const uint8_t *__restrict__ wt1, int64_t n, int dk, int npass, int np, int nkb,
    const float *__restrict__ mcs_g, float x_scale, const float *__restrict__ col_scale,
    float *__restrict__ O, int64_t ldo, int il, float *__restrict__ norms, int64_t nstride,
    float *__restrict__ vmax, const SegCols &segc, int *__restrict__ err, uint64_t wait_ns,
    float norm_limit) {
    using C = Cfg<MODE>;
    constexpr uint32_t SB = stage_bytes<MODE>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + C::STAGES * SB);
    uint64_t *conv = full + C::STAGES;
    uint64_t *empty = conv + C::STAGES;
    uint64_t *accf = empty + C::STAGES;
    uint32_t *tmem_slot = (uint32_t *)(accf + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *nrm_half = (float *)(smem + C::STAGES * SB + kBarArea);        // 128 floats
    float *mcs = (float *)(smem + C::STAGES * SB + kBarArea + 512);       // nkb * BK floats

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = tile * kBM;
    const int col0 = pass * np;

    for (int k = threadIdx.x; k < nkb * C::BK; k += kThreads) mcs[k] = mcs_g[k];
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], kConvWarps / 2);  // one group of converters per block
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(C::TMEM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)tmxp) : "memory");
            const uint32_t tx = (uint32_t)C::XBOX * kXBox + (uint32_t)C::NB * (uint32_t)np * 64u;
            // X boxes kPrefetch K blocks ahead are pulled into L2, so that the
            // stage loads wait on L2 rather than on HBM
            for (int kb = C::STAGES; kb < kPrefetch && kb < nkb; ++kb)
#pragma unroll
                for (int b = 0; b < C::XBOX; ++b) tma_prefetch_2d(tmxp, kb * C::BK + b * 32, (int)row0);
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % C::STAGES;
                const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, err, 1, wait_ns)) break;
                uint8_t *st = smem + s * SB;
                mbar_expect_tx(&full[s], tx);
#pragma unroll
                for (int b = 0; b < C::XBOX; ++b)
                    tma_load_2d(st + b * kXBox, tmxp, kb * C::BK + b * 32, (int)row0, &full[s]);
                uint8_t *bs = st + b_offset<MODE>();
                const int64_t wo = ((int64_t)pass * nkb + kb) * np * 64;
                bulk_load(bs, wt0 + wo, (uint32_t)np * 64u, &full[s]);
                if (C::NB == 2) bulk_load(bs + kBTile, wt1 + wo, (uint32_t)np * 64u, &full[s]);
                if (kb + kPrefetch < nkb)
#pragma unroll
                    for (int b = 0; b < C::XBOX; ++b)
                        tma_prefetch_2d(tmxp, (kb + kPrefetch) * C::BK + b * 32, (int)row0);
                issued = kb + 1;
            }
            // drain: the last loads of each stage must land before the CTA exits
            for (int kb = std::max(0, issued - C::STAGES); kb < issued; ++kb) {
                const int s = kb % C::STAGES;
                const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
                const uint64_t t0 = globaltimer();
                while (!mbar_try(&full[s], ph) && globaltimer() - t0 < kWaitNs) {
                }
            }
        }
    } else if (warp == 1) {
        // The whole warp runs the K loop (warp-uniform control flow and
        // operands, the TMEM base through a warp reduction); one lane, elected
        // inside each instruction, issues the MMAs and commits.
        const uint32_t tmw = __reduce_or_sync(0xffffffffu, tmem);
        const uint32_t idesc = umma_idesc_base<MODE>() | ((uint32_t)(np >> 3) << 17);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % C::STAGES;
            const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
            if (!warp_wait(&conv[s], ph, abort_flag, err, 2, wait_ns)) break;
            tc_fence_after();
            const uint32_t st = smem_u32(smem + s * SB);
            const uint64_t b0 = umma_desc(st + b_offset<MODE>());
            const uint64_t b1 = umma_desc(st + b_offset<MODE>() + kBTile);
            // A of the stage in TMEM, 8 columns per 32-byte K step
            const uint32_t ahi = tmw + ta_col<MODE>(s, 0), alo = tmw + ta_col<MODE>(s, 1);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {  // two 32-byte K steps per 64-byte row
                const uint64_t off = (uint64_t)(kk * 2);
                const uint32_t ka = 8u * (uint32_t)kk;
                umma_ta_elect<MODE>(tmw, ahi + ka, b0 + off, idesc, (kb | kk) != 0);
                if (MODE == kSplit) {
                    umma_ta_elect<MODE>(tmw + kAcc2, ahi + ka, b1 + off, idesc, (kb | kk) != 0);
                    umma_ta_elect<MODE>(tmw + kAcc2, alo + ka, b0 + off, idesc, 1u);
                }
            }
            umma_commit_elect(&empty[s]);
        }
        umma_commit_elect(accf);
        __syncwarp();
    } else {
        // ---- converters: two groups of four warps, group h converting the K
        // blocks kb = h, h + 2, ... (one thread per tile row, the whole block),
        // so that two blocks are converted at once
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const int h = (warp - 2) >> 2;
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);  // the warp's TMEM lane quadrant
        const bool row_ok = row0 + r < n;
        float nrm = 0.f;
        bool ok = true;
        for (int kb = h; kb < nkb && ok; kb += 2) {
            const int s = kb % C::STAGES;
            const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
            int got = 0;
            // The other group may not have consumed this stage's previous block
            // yet; a parity wait cannot tell phase p from phase p + 2, so first
            // wait until the MMAs of block kb - STAGES are done (the stage's
            // barriers are then one phase behind this block at most).
            if (lane == 0)
                got = (kb < C::STAGES || mbar_wait(&empty[s], ph ^ 1u, abort_flag, err, 5, wait_ns)) &&
                              mbar_wait(&full[s], ph, abort_flag, err, 3, wait_ns)
                          ? 1
                          : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) { ok = false; break; }
            uint8_t *st = smem + s * SB;
            const float *mk = mcs + kb * C::BK;
            uint32_t wa[16];  // the row's A values of the stage (split: the hi part)
            uint32_t wl[16];  // split: the lo part
            convert_block<MODE>(st, mk, r, x_scale, nrm, wa, wl);
            // TMEM column c of a buffer holds the row's values of K offsets
            // c * (4 / element bytes) upward, lowest in the low bits
            tmem_st16(tq + ta_col<MODE>(s, 0), wa);
            if (MODE == kSplit) tmem_st16(tq + ta_col<MODE>(s, 1), wl);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[s]);
        }
        // |x - c|^2 of the row: the two groups' partial sums meet in shared memory
        if (h == 1) nrm_half[r] = nrm;
        named_sync(1, 32 * kConvWarps);
        if (h == 0 && pass == 0 && row_ok && ok) {
            const float tot = nrm + nrm_half[r];
            if (norms) norms[(row0 + r) * nstride] = tot / (x_scale * x_scale);
            // |y|^2 >= max_k y_k^2: a row whose scaled, centred squared norm
            // reaches norm_limit may hold a value the operand format cannot
            // represent (the FP16 split overflows at 65504); a non-finite
            // row fails the test too
            if (!(tot < norm_limit)) atomicCAS(err, 0, kErrRange);
        }
        // ---- epilogue: accumulator row r, columns [h * np/2, (h+1) * np/2)
        int ready = 0;
        if (ok && lane == 0) ready = mbar_wait(accf, 0, abort_flag, err, 4, wait_ns) ? 1 : 0;
        ready = __shfl_sync(0xffffffffu, ready, 0);
        if (ready) {
            tc_fence_after();
            tile_epilogue<MODE>(tq, h, 2, lane, r, row0, row_ok, np, col0, dk, col_scale, O, ldo,
                                il, vmax, segc);
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 1) {
        // the accumulator may still be written by MMAs issued before an abort
        if (lane == 0 && *abort_flag) {
            const uint64_t t0 = globaltimer();
            while (!mbar_try(accf, 0) && globaltimer() - t0 < kWaitNs) {
            }
        }
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(C::TMEM)
                     : "memory");
    }
}

// One model's rows: CTA b covers row tile b / npass, column pass b % npass.
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_proj_tc(const __grid_constant__ CUtensorMap tmx, const uint8_t *__restrict__ wt0,
          const uint8_t *__restrict__ wt1, int64_t n, int dk, int npass, int np, int nkb,
          const float *__restrict__ mcs_g, float x_scale, const float *__restrict__ col_scale,
          float *__restrict__ O, int64_t ldo, int il, float *__restrict__ norms,
          int64_t nstride, float *__restrict__ vmax, const SegCols segc,
          int *__restrict__ err, uint64_t wait_ns, float norm_limit) {
    proj_tile<MODE>(&tmx, blockIdx.x / npass, (int)(blockIdx.x % npass), wt0, wt1, n, dk, npass,
                    np, nkb, mcs_g, x_scale, col_scale, O, ldo, il, norms, nstride, vmax, segc,
                    err, wait_ns, norm_limit);
}

// One model's part of a launch: its rows, operands and outputs.
struct ProjGroup {
    CUtensorMap tmx;  // the model's X rows (FP32, 32 x 128 boxes, 128-byte swizzle)
    const uint8_t *wt0, *wt1;
    const float *mcs_g, *col_scale;
    float *O, *norms, *vmax;
    int *err;
    int64_t n, nstride, ldo;
    int dk, npass, np, nkb, il;
    float x_scale, norm_limit;
    SegCols segc;
};
// The tiles of up to kMaxGroups models of one precision (one model for a
// plain encode, a batch of several collections when serving): tile b belongs
// to group g with tile_start[g] <= b < tile_start[g + 1], and within it to
// row tile (b - tile_start[g]) / npass, column pass (b - tile_start[g]) % npass.
struct ProjBatch {
    int ngroups;
    uint64_t wait_ns;
    int64_t tile_start[kMaxGroups + 1];
    ProjGroup g[kMaxGroups];
};

struct TileRef {
    const ProjGroup *P;
    int64_t row0;
    int pass;
};
__device__ __forceinline__ TileRef decode_tile(const ProjBatch &batch, int64_t b) {
    int gi = 0;
    while (gi + 1 < batch.ngroups && b >= batch.tile_start[gi + 1]) ++gi;
    const ProjGroup &P = batch.g[gi];
    const int64_t lb = b - batch.tile_start[gi];
    return TileRef{&P, lb / P.npass * kBM, (int)(lb % P.npass)};
}

// bar.red.or over `threads` threads of named barrier `id`: true in every
// participating thread if v is true in any (a decision all of them take
// alike, so that none waits at a later barrier for one that has left).
__device__ __forceinline__ bool named_any(int id, int threads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(threads)
        : "memory");
    return r != 0;
}

// Named barriers of the converter warps (ids; 0 is __syncthreads).
constexpr int kBarNorm = 1, kBarStop = 2, kBarMcs = 3;

// A persistent CTA: it takes tiles until the batch is done, from the device
// work counter `queue` (one atomicAdd per tile) or, without one, tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Tile t of the CTA goes through a
// ring of slots in shared memory (two; four with DB): the producer fetches it
// and publishes it (tile_full), every other role reads it and releases the
// slot (tile_empty).  Every role keeps one running K-block counter `it` over
// all of its tiles, so that the stage barriers' phases run on from tile to
// tile and the producer loads the next tile's first stages while the
// previous tile is still being drained.
// Without DB the converter warps also drain the one accumulator, and the
// MMA warp starts the next tile's MMAs once every converter warp has read it
// (acc_empty).  With DB (BF16 / FP8, passes of at most kAccDb columns) tile t
// accumulates into accumulator t % 2 and four more warps drain it, so that
// its epilogue runs beside tile t + 1's MMAs; the MMA warp waits only for the
// epilogue of tile t - 1 (acc_empty[t % 2]).
template <int MODE, bool DB>
__device__ __forceinline__ void proj_persistent(const ProjBatch &batch, int *queue) {
    using C = Cfg<MODE>;
    constexpr uint32_t SB = stage_bytes<MODE>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + C::STAGES * SB);
    uint64_t *conv = full + C::STAGES;
    uint64_t *empty = conv + C::STAGES;
    constexpr int R = DB ? 4 : 2;     // tile ring slots
    constexpr int NACC = DB ? 2 : 1;  // accumulators
    uint64_t *accf = empty + C::STAGES;       // NACC: an accumulator's MMAs are complete
    uint64_t *tile_full = accf + NACC;         // R
    uint64_t *tile_empty = tile_full + R;      // R
    uint64_t *acc_empty = tile_empty + R;      // NACC: an accumulator has been read
    uint64_t *mma_done = acc_empty + NACC;     // every MMA issued is complete (at exit)
    int64_t *ring = (int64_t *)(mma_done + 1);  // R
    uint32_t *tmem_slot = (uint32_t *)(ring + R);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    float *nrm_half = (float *)(smem + C::STAGES * SB + kBarArea);   // 128 floats
    float *mcs = (float *)(smem + C::STAGES * SB + kBarArea + 512);  // nkb * BK floats

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t total = batch.tile_start[batch.ngroups];
    const uint64_t wait_ns = batch.wait_ns;
    // the error word of the first group takes the bounded waits' codes
    int *err = batch.g[0].err;

    {
        const ProjGroup &P0 = batch.g[0];
        for (int k = threadIdx.x; k < P0.nkb * C::BK; k += (int)blockDim.x) mcs[k] = P0.mcs_g[k];
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], kConvWarps / 2);  // one group of converters per block
            mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(&accf[i], 1);
            // read by every converter warp (one accumulator) or every epilogue warp
            mbar_init(&acc_empty[i], DB ? kEpiWarps : kConvWarps);
        }
        for (int i = 0; i < R; ++i) {
            mbar_init(&tile_full[i], 1);
            // the MMA warp, every converter warp and every epilogue warp
            mbar_init(&tile_empty[i], 1 + kConvWarps + (DB ? kEpiWarps : 0));
        }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(C::TMEM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;  // K blocks issued over all tiles
            for (int t = 0;; ++t) {
                const int slot = t % R;
                // the slot's tile t - R has been read by every consumer
                if (t >= R &&
                    !mbar_wait(&tile_empty[slot], (uint32_t)(t / R - 1) & 1u, abort_flag, err, 1,
                               wait_ns))
                    break;
                int64_t b = queue ? (int64_t)atomicAdd(queue, 1)
                                  : (int64_t)blockIdx.x + (int64_t)t * gridDim.x;
                if (b >= total) b = -1;
                ring[slot] = b;
                mbar_arrive(&tile_full[slot]);
                if (b < 0) break;
                const TileRef tr = decode_tile(batch, b);
                const ProjGroup &P = *tr.P;
                const CUtensorMap *tmxp = &P.tmx;
                // the tile's fields in registers: a read through the batch
                // reference would be repeated after every asm with a memory
                // clobber in the loop
                const uint8_t *wt0 = P.wt0, *wt1 = P.wt1;
                const int np = P.np;
                asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)tmxp) : "memory");
                const uint32_t tx =
                    (uint32_t)C::XBOX * kXBox + (uint32_t)C::NB * (uint32_t)np * 64u;
                const int nkb = P.nkb;
                const int row0 = (int)tr.row0;
                // X boxes kPrefetch K blocks ahead are pulled into L2, so that
                // the stage loads wait on L2 rather than on HBM
                for (int kb = C::STAGES; kb < kPrefetch && kb < nkb; ++kb)
#pragma unroll
                    for (int bx = 0; bx < C::XBOX; ++bx)
                        tma_prefetch_2d(tmxp, kb * C::BK + bx * 32, row0);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % (uint32_t)C::STAGES);
                    const uint32_t ph = (it / (uint32_t)C::STAGES) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, err, 1, wait_ns)) {
                        ok = false;
                        break;
                    }
                    uint8_t *st = smem + s * SB;
                    mbar_expect_tx(&full[s], tx);
#pragma unroll
                    for (int bx = 0; bx < C::XBOX; ++bx)
                        tma_load_2d(st + bx * kXBox, tmxp, kb * C::BK + bx * 32, row0, &full[s]);
                    uint8_t *bs = st + b_offset<MODE>();
                    const int64_t wo = ((int64_t)tr.pass * nkb + kb) * np * 64;
                    bulk_load(bs, wt0 + wo, (uint32_t)np * 64u, &full[s]);
                    if (C::NB == 2) bulk_load(bs + kBTile, wt1 + wo, (uint32_t)np * 64u, &full[s]);
                    if (kb + kPrefetch < nkb)
#pragma unroll
                        for (int bx = 0; bx < C::XBOX; ++bx)
                            tma_prefetch_2d(tmxp, (kb + kPrefetch) * C::BK + bx * 32, row0);
                }
                if (!ok) break;
            }
            // drain: the last loads of each stage must land before the CTA exits
            for (uint32_t i = it > (uint32_t)C::STAGES ? it - (uint32_t)C::STAGES : 0u; i < it; ++i) {
                const int s = (int)(i % (uint32_t)C::STAGES);
                const uint32_t ph = (i / (uint32_t)C::STAGES) & 1u;
                const uint64_t t0 = globaltimer();
                while (!mbar_try(&full[s], ph) && globaltimer() - t0 < kWaitNs) {
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // The whole warp runs the MMA loop, so that its control flow and the
        // operands of the tcgen05 instructions are warp-uniform; one lane,
        // elected inside each instruction, issues the MMAs and commits.
        // the TMEM base and each tile number through a warp reduction: values
        // the compiler then treats as warp-uniform
        const uint32_t tmw = __reduce_or_sync(0xffffffffu, tmem);
        uint32_t it = 0;       // K blocks consumed over all tiles
        uint32_t commits = 0;  // accumulator commits issued (one per tile)
        bool ok = true;
        for (int t = 0; ok; ++t) {
            const int slot = t % R;
            if (!warp_wait(&tile_full[slot], (uint32_t)(t / R) & 1u, abort_flag, err, 2, wait_ns))
                break;
            const int64_t b = (int64_t)__reduce_max_sync(0xffffffffu, (int)ring[slot]);
            if (lane == 0) mbar_arrive(&tile_empty[slot]);
            if (b < 0) break;
            const TileRef tr = decode_tile(batch, b);
            const ProjGroup &P = *tr.P;
            const uint32_t idesc = umma_idesc_base<MODE>() | ((uint32_t)(P.np >> 3) << 17);
            const int nkb = P.nkb;
            // tile t's accumulator (DB: the two alternate) is free once its
            // previous tile has been read
            const int a = DB ? (t & 1) : 0;
            const uint32_t dacc = tmw + (uint32_t)a * kAccDb;
            if (DB ? (t >= 2 && !warp_wait(&acc_empty[a], (uint32_t)((t >> 1) - 1) & 1u, abort_flag,
                                           err, 2, wait_ns))
                   : (t >= 1 && !warp_wait(acc_empty, (uint32_t)(t - 1) & 1u, abort_flag, err, 2,
                                           wait_ns)))
                break;
            tc_fence_after();
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                const int s = (int)(it % (uint32_t)C::STAGES);
                const uint32_t ph = (it / (uint32_t)C::STAGES) & 1u;
                if (!warp_wait(&conv[s], ph, abort_flag, err, 2, wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t st = smem_u32(smem + s * SB);
                const uint64_t b0 = umma_desc(st + b_offset<MODE>());
                const uint64_t b1 = umma_desc(st + b_offset<MODE>() + kBTile);
                // A of the stage in TMEM, 8 columns per 32-byte K step
                const uint32_t ahi = tmw + (DB ? kTADb + 16u * (uint32_t)s : ta_col<MODE>(s, 0));
                const uint32_t alo = tmw + ta_col<MODE>(s, 1);
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {  // two 32-byte K steps per 64-byte row
                    const uint64_t off = (uint64_t)(kk * 2);
                    const uint32_t ka = 8u * (uint32_t)kk;
                    umma_ta_elect<MODE>(dacc, ahi + ka, b0 + off, idesc, (kb | kk) != 0);
                    if (MODE == kSplit) {
                        umma_ta_elect<MODE>(tmw + kAcc2, ahi + ka, b1 + off, idesc, (kb | kk) != 0);
                        umma_ta_elect<MODE>(tmw + kAcc2, alo + ka, b0 + off, idesc, 1u);
                    }
                }
                umma_commit_elect(&empty[s]);
            }
            // the tile's accumulator (after an abort: every MMA issued so far)
            umma_commit_elect(&accf[a]);
            ++commits;
        }
        // at exit every MMA issued must be complete before TMEM is freed
        if (commits > 0) {
            umma_commit_elect(mma_done);
            if (lane == 0) {
                const uint64_t t0 = globaltimer();
                while (!mbar_try(mma_done, 0) && globaltimer() - t0 < kWaitNs) {
                }
            }
        }
        __syncwarp();
    } else if (warp < 2 + kConvWarps) {
        // ---- converters: two groups of four warps, group h converting the K
        // blocks kb = h, h + 2, ... of each tile (one thread per tile row, the
        // whole block), so that two blocks are converted at once; then the
        // tile's epilogue
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const int h = (warp - 2) >> 2;
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);  // the warp's TMEM lane quadrant
        uint32_t base = 0;  // K blocks of this CTA's earlier tiles
        // the first group's -c * s is in shared memory from the prologue
        const ProjGroup *gcur = &batch.g[0];
        bool ok = true;
        for (int t = 0;; ++t) {
            const int slot = t % R;
            int got = 0;
            long long bl = -1;
            if (lane == 0) {
                got = mbar_wait(&tile_full[slot], (uint32_t)(t / R) & 1u, abort_flag, err, 3, wait_ns)
                          ? 1
                          : 0;
                if (got) {
                    bl = ring[slot];
                    mbar_arrive(&tile_empty[slot]);
                }
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            const int64_t b = (int64_t)__shfl_sync(0xffffffffu, bl, 0);
            // the converter warps stop together (the end of the work, or a
            // failed wait in any of them)
            if (named_any(kBarStop, 32 * kConvWarps, !ok || !got || b < 0)) break;
            const TileRef tr = decode_tile(batch, b);
            const ProjGroup &P = *tr.P;
            const int64_t row0 = tr.row0;
            const int pass = tr.pass, nkb = P.nkb, np = P.np, dk = P.dk;
            const float x_scale = P.x_scale;
            const int col0 = pass * np;
            if (tr.P != gcur) {
                // the model's -c * s into shared memory (every converter warp
                // is past its conversions of the earlier tiles)
                for (int k = (int)threadIdx.x - 64; k < nkb * C::BK; k += 32 * kConvWarps)
                    mcs[k] = P.mcs_g[k];
                named_sync(kBarMcs, 32 * kConvWarps);
                gcur = tr.P;
            }
            const bool row_ok = row0 + r < P.n;
            float nrm = 0.f;
            for (int kb = h; kb < nkb && ok; kb += 2) {
                const uint32_t it = base + (uint32_t)kb;
                const int s = (int)(it % (uint32_t)C::STAGES);
                const uint32_t ph = (it / (uint32_t)C::STAGES) & 1u;
                int gotk = 0;
                // The other group may not have consumed this stage's previous
                // block yet; a parity wait cannot tell phase p from phase p + 2,
                // so first wait until the MMAs of block it - STAGES are done
                // (the stage's barriers are then one phase behind this block at
                // most).
                if (lane == 0)
                    gotk = (it < (uint32_t)C::STAGES ||
                            mbar_wait(&empty[s], ph ^ 1u, abort_flag, err, 5, wait_ns)) &&
                                   mbar_wait(&full[s], ph, abort_flag, err, 3, wait_ns)
                               ? 1
                               : 0;
                gotk = __shfl_sync(0xffffffffu, gotk, 0);
                if (!gotk) {
                    ok = false;
                    break;
                }
                uint8_t *st = smem + s * SB;
                const float *mk = mcs + kb * C::BK;
                uint32_t wa[16];  // the row's A values of the stage (split: the hi part)
                uint32_t wl[16];  // split: the lo part
                convert_block<MODE>(st, mk, r, x_scale, nrm, wa, wl);
                // TMEM column c of a buffer holds the row's values of K offsets
                // c * (4 / element bytes) upward, lowest in the low bits
                tmem_st16(tq + (DB ? kTADb + 16u * (uint32_t)s : ta_col<MODE>(s, 0)), wa);
                if (MODE == kSplit) tmem_st16(tq + ta_col<MODE>(s, 1), wl);
                tmem_st_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&conv[s]);
            }
            // |x - c|^2 of the row: the two groups' partial sums meet in shared memory
            if (h == 1) nrm_half[r] = nrm;
            named_sync(kBarNorm, 32 * kConvWarps);
            if (h == 0 && pass == 0 && row_ok && ok) {
                const float tot = nrm + nrm_half[r];
                if (P.norms) P.norms[(row0 + r) * P.nstride] = tot / (x_scale * x_scale);
                // |y|^2 >= max_k y_k^2: a row whose scaled, centred squared norm
                // reaches norm_limit may hold a value the operand format cannot
                // represent (the FP16 split overflows at 65504); a non-finite
                // row fails the test too
                if (!(tot < P.norm_limit)) atomicCAS(P.err, 0, kErrRange);
            }
            if constexpr (!DB) {
                // ---- epilogue: accumulator row r, 32-column blocks h, h + 2, ...
                int ready = 0;
                if (ok && lane == 0)
                    ready = mbar_wait(accf, (uint32_t)t & 1u, abort_flag, err, 4, wait_ns) ? 1 : 0;
                ready = __shfl_sync(0xffffffffu, ready, 0);
                if (!ready) ok = false;
                if (ready) {
                    tc_fence_after();
                    tile_epilogue<MODE>(tq, h, 2, lane, r, row0, row_ok, np, col0, dk, P.col_scale,
                                        P.O, P.ldo, P.il, P.vmax, P.segc);
                }
                // the accumulator may take the next tile's MMAs once every
                // converter warp has read it
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
            }
            base += (uint32_t)nkb;
        }
        tc_fence_before();
    } else {
        if constexpr (DB) {
            // ---- epilogue warps (DB): warp w drains TMEM lane quadrant w % 4,
            // every 32-column block of tile t's accumulator t % 2, while the
            // MMA warp fills the other one
            const int q = warp & 3;
            const int r = q * 32 + lane;
            const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
            for (int t = 0;; ++t) {
                const int slot = t % R;
                int got = 0;
                long long bl = -1;
                if (lane == 0) {
                    got = mbar_wait(&tile_full[slot], (uint32_t)(t / R) & 1u, abort_flag, err, 4,
                                    wait_ns)
                              ? 1
                              : 0;
                    if (got) {
                        bl = ring[slot];
                        mbar_arrive(&tile_empty[slot]);
                    }
                }
                got = __shfl_sync(0xffffffffu, got, 0);
                const int64_t b = (int64_t)__shfl_sync(0xffffffffu, bl, 0);
                if (!got || b < 0) break;
                const TileRef tr = decode_tile(batch, b);
                const ProjGroup &P = *tr.P;
                const int a = t & 1;
                int ready = 0;
                if (lane == 0)
                    ready = mbar_wait(&accf[a], (uint32_t)(t >> 1) & 1u, abort_flag, err, 4, wait_ns)
                                ? 1
                                : 0;
                ready = __shfl_sync(0xffffffffu, ready, 0);
                if (!ready) break;
                tc_fence_after();
                const int np = P.np;
                tile_epilogue<MODE>(tq + (uint32_t)a * kAccDb, 0, 1, lane, r, tr.row0,
                                    tr.row0 + r < P.n, np, tr.pass * np, P.dk, P.col_scale, P.O,
                                    P.ldo, P.il, P.vmax, P.segc);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[a]);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(C::TMEM)
                     : "memory");
    }
}

// Persistent projection of a serving batch: one CTA per SM, each taking tiles
// of the batch until it is done (queue: the device work counter, zero at
// launch; NULL: the static order blockIdx.x, blockIdx.x + gridDim.x, ...).
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_proj_tc_persistent(const __grid_constant__ ProjBatch batch, int *queue) {
    proj_persistent<MODE, false>(batch, queue);
}
// The double-buffered form (BF16): two accumulators of at most kAccDb
// columns and four epilogue warps, so that a tile's epilogue overlaps the
// next tile's MMAs.
template <int MODE>
__global__ void __launch_bounds__(kThreadsDb, 1)
k_proj_tc_db(const __grid_constant__ ProjBatch batch, int *queue) {
    proj_persistent<MODE, true>(batch, queue);
}

// ------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

saq_status get_encoder(PFN_cuTensorMapEncodeTiled_v12000 *fn) {
    std::call_once(g_encode_once, []() {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    if (!g_encode) return set_error(SAQ_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    *fn = g_encode;
    return SAQ_OK;
}

saq_status make_map(CUtensorMap *map, CUtensorMapDataType type, int elem, const void *ptr,
                    uint64_t inner, uint64_t outer, uint32_t box_inner, uint32_t box_outer,
                    CUtensorMapSwizzle swz) {
    PFN_cuTensorMapEncodeTiled_v12000 enc;
    saq_status st = get_encoder(&enc);
    if (st != SAQ_OK) return st;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * (uint64_t)elem};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(map, type, 2, const_cast<void *>(ptr), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(SAQ_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return SAQ_OK;
}

struct TcExtra {
    float *mcs = nullptr;  // -c * x_scale, padded to the K blocks
    float x_scale = 1.f;
    int np = 0, npass = 0;
    int *err = nullptr;
    bool db = false;  // BF16 / FP8 on the double-buffered kernel (passes of at most kAccDb)
};

double pow2_near(double x) { return ldexp(1.0, (int)lround(log2(x))); }

// W operand (dkpad rows x dpad values, K-major) cut into the tiles the kernel
// copies whole: tile (pass p, K block kb) holds rows p*np .. p*np + np - 1,
// values kb*bk .. kb*bk + bk - 1, one 64-byte row each, with the 16-byte
// chunks of row r permuted as the MMA's 64-byte swizzle expects
// (chunk c at r * 64 + ((c ^ ((r >> 1) & 3)) * 16)).
template <typename T>
std::vector<T> tile_operand(const std::vector<T> &w, int dkpad, int dpad, int np, int bk) {
    static_assert(sizeof(T) == 1 || sizeof(T) == 2, "operand element of 1 or 2 bytes");
    constexpr int per_chunk = 16 / (int)sizeof(T);
    const int npass = dkpad / np, nkb = dpad / bk;
    std::vector<T> t(w.size());
    for (int p = 0; p < npass; ++p)
        for (int kb = 0; kb < nkb; ++kb)
            for (int r = 0; r < np; ++r)
                for (int c = 0; c < 4; ++c) {
                    const size_t dst = (((size_t)p * nkb + kb) * np * 64 + (size_t)r * 64 +
                                        (size_t)((c ^ ((r >> 1) & 3)) * 16)) / sizeof(T);
                    const size_t src = ((size_t)p * np + r) * dpad + (size_t)kb * bk + (size_t)c * per_chunk;
                    for (int e = 0; e < per_chunk; ++e) t[dst + e] = w[src + e];
                }
    return t;
}

// Role-wait bound of the next launches (saq_set_wait_limit).
std::atomic<uint64_t> g_wait_ns{kWaitNs};

template <int MODE> saq_status launch_mode(const saq_model *m, const float *X, int64_t n,
                                           float *O, int64_t ldo, int layout, float *norms,
                                           int64_t ns, float *vmax, int *err, cudaStream_t s) {
    const TcExtra *ex = static_cast<const TcExtra *>(m->tc.extra);
    // |y|^2 bound of a row (y = (x - c) s): the FP16 split overflows past
    // 65504; BF16 and E4M3 (saturating) only flag non-finite rows
    const float norm_limit = MODE == kSplit ? 65504.f * 65504.f : INFINITY;
    CUtensorMap tmx;
    saq_status st = make_map(&tmx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, X, (uint64_t)m->d,
                             (uint64_t)n, 32, kBM, CU_TENSOR_MAP_SWIZZLE_128B);
    if (st != SAQ_OK) return st;
    const int nkb = m->tc.d_pad / Cfg<MODE>::BK;
    const uint32_t sm = smem_bytes<MODE>(m->tc.d_pad);
    SAQ_CUDA_CHECK(cudaFuncSetAttribute(k_proj_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sm));
    const int64_t tiles = (n + kBM - 1) / kBM;
    const int64_t blocks = tiles * ex->npass;
    if (blocks > 0x7FFFFFFF) return set_error(SAQ_ERR_UNSUPPORTED, "too many rows in one call");
    {
        LaunchTimer lt_(kKindProject, s);
        k_proj_tc<MODE><<<(unsigned)blocks, kThreads, sm, s>>>(
            tmx, (const uint8_t *)m->tc.w_hi,
            (const uint8_t *)(m->tc.w_lo ? m->tc.w_lo : m->tc.w_hi), n, m->dk, ex->npass, ex->np, nkb, ex->mcs, ex->x_scale,
            m->tc.col_scale, O, ldo, layout == kInterleaved ? 1 : 0, norms, ns, vmax, seg_cols(m),
            err ? err : ex->err, g_wait_ns.load(), norm_limit);
    }
    note_launches();
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

}  // namespace

// d % 4 == 0 for the FP32 tensor map; the -c*s copy of the K range must fit
// in shared memory next to the stages.
bool tc_supported(const saq_model *m) { return m->d % 4 == 0 && m->dk > 0 && m->d <= 6144; }

void tc_release(saq_model *m) {
    TcExtra *ex = static_cast<TcExtra *>(m->tc.extra);
    if (ex) {
        cudaFree(ex->mcs);
        cudaFree(ex->err);
        delete ex;
    }
    cudaFree(m->tc.w_hi);
    cudaFree(m->tc.w_lo);
    cudaFree(m->tc.col_scale);
    m->tc = TcOperands{};
}

// Device operands of W for `precision`: zero-padded to dk_pad x d_pad, the
// per-column dequantisation scale, and -c * x_scale for the centring FMA.
saq_status model_build_tc(saq_model *m, int precision, cudaStream_t) {
    if (!tc_supported(m))
        return set_error(SAQ_ERR_UNSUPPORTED, "tensor-core projection needs d %% 4 == 0, d <= 6144");
    tc_release(m);
    const int BK = precision == SAQ_PREC_FP8 ? 64 : 32;
    const int dpad = (m->d + BK - 1) / BK * BK;
    const int d = m->d, dk = m->dk;
    // balanced column passes of at most 256 columns (split: 192), multiples
    // of 16.  BF16 and FP8 run on the double-buffered kernel, whose two
    // accumulators hold at most kAccDb columns each, when the tiles are short
    // (d <= 1024: the hidden epilogue is a large share of a tile) and the
    // narrower passes are at most a quarter more.  Measured against the
    // per-tile kernel: d = 960, five passes instead of four, BF16 9% and FP8
    // 15% faster; BF16 at d = 1536 (eight instead of six) 11% slower; FP8 at
    // d = 3072 (ten instead of eight, 15 instead of 12) equal and 13% slower.
    const int p256 = (dk + kNPMax - 1) / kNPMax, pdb = (dk + (int)kAccDb - 1) / (int)kAccDb;
    const bool db = (precision == SAQ_PREC_BF16 || precision == SAQ_PREC_FP8) && d <= 1024 &&
                    4 * pdb <= 5 * p256;
    const int npmax = precision == SAQ_PREC_FP32 ? kSplitNP : db ? (int)kAccDb : kNPMax;
    const int npass = (dk + npmax - 1) / npmax;
    const int np = ((dk + npass - 1) / npass + 15) / 16 * 16;
    const int dkpad = npass * np;
    // input scale from the fitted variances (a power of two: exact)
    double tot = 0;
    for (double v : m->sig2) tot += v;
    const double rms = tot > 0 ? sqrt(tot / d) : 0.0;
    double xs = 1.0, ws = 1.0;
    std::vector<float> cs((size_t)dkpad, 0.f);
    TcExtra *ex = new TcExtra();
    m->tc.extra = ex;
    m->tc.precision = precision;
    m->tc.dk_pad = dkpad;
    m->tc.d_pad = dpad;
    ex->np = np;
    ex->npass = npass;
    ex->db = db;
    if (precision == SAQ_PREC_FP32) {
        xs = rms > 0 ? pow2_near(8.0 / rms) : 1.0;
        ws = 1024.0;
        std::vector<__half> hi((size_t)dkpad * dpad, __float2half(0.f)), lo = hi;
        for (int i = 0; i < dk; ++i)
            for (int k = 0; k < d; ++k) {
                const double w = m->W[(size_t)i * d + k] * ws;
                const __half h = __double2half(w);
                hi[(size_t)i * dpad + k] = h;
                lo[(size_t)i * dpad + k] = __double2half(w - (double)__half2float(h));
            }
        hi = tile_operand(hi, dkpad, dpad, np, BK);
        lo = tile_operand(lo, dkpad, dpad, np, BK);
        SAQ_CUDA_CHECK(cudaMalloc(&m->tc.w_hi, hi.size() * 2));
        SAQ_CUDA_CHECK(cudaMalloc(&m->tc.w_lo, lo.size() * 2));
        SAQ_CUDA_CHECK(cudaMemcpy(m->tc.w_hi, hi.data(), hi.size() * 2, cudaMemcpyHostToDevice));
        SAQ_CUDA_CHECK(cudaMemcpy(m->tc.w_lo, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice));
        for (int i = 0; i < dk; ++i) cs[(size_t)i] = (float)(1.0 / (xs * ws));
    } else if (precision == SAQ_PREC_BF16) {
        std::vector<__nv_bfloat16> b((size_t)dkpad * dpad, __float2bfloat16(0.f));
        for (int i = 0; i < dk; ++i)
            for (int k = 0; k < d; ++k)
                b[(size_t)i * dpad + k] = __float2bfloat16((float)m->W[(size_t)i * d + k]);
        b = tile_operand(b, dkpad, dpad, np, BK);
        SAQ_CUDA_CHECK(cudaMalloc(&m->tc.w_hi, b.size() * 2));
        SAQ_CUDA_CHECK(cudaMemcpy(m->tc.w_hi, b.data(), b.size() * 2, cudaMemcpyHostToDevice));
        for (int i = 0; i < dk; ++i) cs[(size_t)i] = 1.f;
    } else if (precision == SAQ_PREC_FP8) {
        // E4M3: inputs scaled so the per-coordinate rms maps to 16 (max 448),
        // each kept segment's rows scaled by a power of two so |w| <= 448.
        xs = rms > 0 ? pow2_near(16.0 / rms) : 1.0;
        std::vector<uint8_t> b((size_t)dkpad * dpad, 0);
        for (const KeptSeg &k : m->kept) {
            double amax = 0;
            for (int i = k.off; i < k.off + k.len; ++i)
                for (int j = 0; j < d; ++j) amax = std::max(amax, fabs(m->W[(size_t)i * d + j]));
            const double sb = amax > 0 ? ldexp(1.0, (int)floor(log2(448.0 / amax))) : 1.0;
            for (int i = k.off; i < k.off + k.len; ++i) {
                for (int j = 0; j < d; ++j)
                    b[(size_t)i * dpad + j] = (uint8_t)__nv_cvt_double_to_fp8(
                        m->W[(size_t)i * d + j] * sb, __NV_SATFINITE, __NV_E4M3);
                cs[(size_t)i] = (float)(1.0 / (xs * sb));
            }
        }
        b = tile_operand(b, dkpad, dpad, np, BK);
        SAQ_CUDA_CHECK(cudaMalloc(&m->tc.w_hi, b.size()));
        SAQ_CUDA_CHECK(cudaMemcpy(m->tc.w_hi, b.data(), b.size(), cudaMemcpyHostToDevice));
    } else {
        return set_error(SAQ_ERR_INVALID, "precision %d has no tensor-core form", precision);
    }
    ex->x_scale = (float)xs;
    cs.resize(cs.size() + 256, 0.f);  // the epilogue reads whole 32-column blocks
    SAQ_CUDA_CHECK(cudaMalloc(&m->tc.col_scale, sizeof(float) * cs.size()));
    SAQ_CUDA_CHECK(cudaMemcpy(m->tc.col_scale, cs.data(), sizeof(float) * cs.size(),
                              cudaMemcpyHostToDevice));
    // -c * s, exact (s is a power of two); y = fma(x, s, -c*s) = round((x - c) s)
    std::vector<float> mp((size_t)dpad, 0.f);
    for (int k = 0; k < d; ++k) mp[(size_t)k] = -(float)m->mean[(size_t)k] * (float)xs;
    SAQ_CUDA_CHECK(cudaMalloc(&ex->mcs, sizeof(float) * mp.size()));
    SAQ_CUDA_CHECK(cudaMemcpy(ex->mcs, mp.data(), sizeof(float) * mp.size(), cudaMemcpyHostToDevice));
    SAQ_CUDA_CHECK(cudaMalloc(&ex->err, sizeof(int)));
    SAQ_CUDA_CHECK(cudaMemset(ex->err, 0, sizeof(int)));
    return SAQ_OK;
}

SegCols seg_cols(const saq_model *m) {
    SegCols c{};
    c.nk = (int32_t)m->kept.size();
    for (int i = 0; i < 64; ++i) c.end[i] = 0x7fffffff;
    for (int i = 0; i < c.nk && i < 64; ++i) c.end[i] = m->kept[(size_t)i].off + m->kept[(size_t)i].len;
    return c;
}

namespace {
template <int MODE>
saq_status launch_persistent_single(const saq_model *m, const float *X, int64_t n, float *O,
                                    int64_t ldo, int il, float *norms, int64_t ns, float *vmax,
                                    int *err, bool db, cudaStream_t s);
}  // namespace

saq_status launch_project_tc(const saq_model *m, const float *X, int64_t n, float *O,
                             int64_t ldo, int layout, float *norms2, int64_t norms_stride,
                             float *vmax, int *err, cudaStream_t s) {
    if (n <= 0) return SAQ_OK;
    if (((uintptr_t)X & 15u) != 0) return set_error(SAQ_ERR_INVALID, "X not 16-byte aligned");
    if (m->kept.size() > 64) return set_error(SAQ_ERR_UNSUPPORTED, "more than 64 kept segments");
    switch (m->tc.precision) {
        case SAQ_PREC_FP32:
            // the persistent kernel (start-up and CTA changes hidden: 1.8%
            // faster than a CTA per tile at d = 960)
            return launch_persistent_single<kSplit>(m, X, n, O, ldo, layout == kInterleaved ? 1 : 0,
                                                    norms2, norms_stride, vmax, err, false, s);
        case SAQ_PREC_BF16:
            // the double-buffered persistent kernel where the model's passes
            // allow it, else a CTA per tile (the persistent form without the
            // second accumulator measured slower for the long tiles left)
            if (static_cast<const TcExtra *>(m->tc.extra)->db)
                return launch_persistent_single<kBF16>(m, X, n, O, ldo,
                                                       layout == kInterleaved ? 1 : 0, norms2,
                                                       norms_stride, vmax, err, true, s);
            return launch_mode<kBF16>(m, X, n, O, ldo, layout, norms2, norms_stride, vmax, err, s);
        case SAQ_PREC_FP8:
            if (static_cast<const TcExtra *>(m->tc.extra)->db)
                return launch_persistent_single<kFP8>(m, X, n, O, ldo,
                                                      layout == kInterleaved ? 1 : 0, norms2,
                                                      norms_stride, vmax, err, true, s);
            return launch_mode<kFP8>(m, X, n, O, ldo, layout, norms2, norms_stride, vmax, err, s);
    }
    return set_error(SAQ_ERR_INVALID, "tensor-core operands not built");
}

namespace {
// Operands and outputs of model m's rows X (n) as one group of a persistent
// launch (interleaved output with v_max, |x - c|^2 into norms).
template <int MODE>
saq_status fill_group(ProjGroup *g, const ProjJob &j, int64_t ldo, int il) {
    const saq_model *m = j.m;
    const TcExtra *ex = static_cast<const TcExtra *>(m->tc.extra);
    saq_status st = make_map(&g->tmx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, j.X, (uint64_t)m->d,
                             (uint64_t)j.n, 32, kBM, CU_TENSOR_MAP_SWIZZLE_128B);
    if (st != SAQ_OK) return st;
    g->wt0 = (const uint8_t *)m->tc.w_hi;
    g->wt1 = (const uint8_t *)(m->tc.w_lo ? m->tc.w_lo : m->tc.w_hi);
    g->mcs_g = ex->mcs;
    g->col_scale = m->tc.col_scale;
    g->O = j.O;
    g->norms = j.norms;
    g->vmax = j.vmax;
    g->err = j.err ? j.err : ex->err;
    g->n = j.n;
    g->nstride = j.nstride;
    g->ldo = ldo;
    g->il = il;
    g->dk = m->dk;
    g->npass = ex->npass;
    g->np = ex->np;
    g->nkb = m->tc.d_pad / Cfg<MODE>::BK;
    g->x_scale = ex->x_scale;
    g->norm_limit = MODE == kSplit ? 65504.f * 65504.f : INFINITY;
    g->segc = seg_cols(m);
    return SAQ_OK;
}

// SMs of the current device (one persistent CTA each).
int sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev < 64 && cached[dev].load() > 0) return cached[dev].load();
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    if (dev < 64) cached[dev].store(sms);
    return sms;
}

// The batch's tiles on one persistent CTA per SM (at most one per tile), taken
// in order from the work counter: the column passes of a row tile,
// consecutive tiles, run at about the same time and share X in L2.  BF16
// runs the double-buffered kernel when every group's passes fit its
// accumulators (db).
template <int MODE>
saq_status launch_persistent(const ProjBatch &b, int dpad_max, int *queue, bool db,
                             cudaStream_t s) {
    const int64_t tiles = b.tile_start[b.ngroups];
    if (tiles <= 0) return SAQ_OK;
    if (tiles > 0x7FFFFFFF) return set_error(SAQ_ERR_UNSUPPORTED, "too many rows in one call");
    const uint32_t sm = smem_bytes<MODE>(dpad_max);
    const int64_t grid = std::min<int64_t>(tiles, sm_count());
    if constexpr (MODE != kSplit) {
        if (db) {
            SAQ_CUDA_CHECK(cudaFuncSetAttribute(k_proj_tc_db<MODE>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            {
                LaunchTimer lt_(kKindProject, s);
                k_proj_tc_db<MODE><<<(unsigned)grid, kThreadsDb, sm, s>>>(b, queue);
            }
            note_launches();
            SAQ_CUDA_CHECK(cudaGetLastError());
            return SAQ_OK;
        }
    }
    SAQ_CUDA_CHECK(cudaFuncSetAttribute(k_proj_tc_persistent<MODE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    {
        LaunchTimer lt_(kKindProject, s);
        k_proj_tc_persistent<MODE><<<(unsigned)grid, kThreads, sm, s>>>(b, queue);
    }
    note_launches();
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

template <int MODE>
saq_status launch_grouped_mode(const ProjJob *jobs, int njobs, int *queue, cudaStream_t s) {
    ProjBatch b;
    memset(&b, 0, sizeof(b));
    b.wait_ns = g_wait_ns.load();
    b.tile_start[0] = 0;
    int dpad_max = 0;
    bool db = true;
    for (int i = 0; i < njobs; ++i) {
        const ProjJob &j = jobs[i];
        const saq_model *m = j.m;
        if (j.n <= 0 || m->dk == 0) continue;
        const TcExtra *ex = static_cast<const TcExtra *>(m->tc.extra);
        db = db && ex->np <= (int)kAccDb;
        saq_status st = fill_group<MODE>(&b.g[b.ngroups], j, m->dk, 1);
        if (st != SAQ_OK) return st;
        dpad_max = std::max(dpad_max, m->tc.d_pad);
        b.tile_start[b.ngroups + 1] = b.tile_start[b.ngroups] + (j.n + kBM - 1) / kBM * ex->npass;
        ++b.ngroups;
    }
    if (b.ngroups == 0) return SAQ_OK;
    const int64_t tiles = b.tile_start[b.ngroups];
    if (tiles > 0x7FFFFFFF) return set_error(SAQ_ERR_UNSUPPORTED, "too many rows in one call");
    return launch_persistent<MODE>(b, dpad_max, queue, db, s);
}

// One model's rows on the persistent kernel (db: the double-buffered one),
// with a work counter of its own from the stream-ordered pool (freed after
// the launch on s).
template <int MODE>
saq_status launch_persistent_single(const saq_model *m, const float *X, int64_t n, float *O,
                                    int64_t ldo, int il, float *norms, int64_t ns, float *vmax,
                                    int *err, bool db, cudaStream_t s) {
    const TcExtra *ex = static_cast<const TcExtra *>(m->tc.extra);
    ProjBatch b;
    memset(&b, 0, sizeof(b));
    b.ngroups = 1;
    b.wait_ns = g_wait_ns.load();
    saq_status st =
        fill_group<MODE>(&b.g[0], ProjJob{m, X, n, O, norms, ns, vmax, err}, ldo, il);
    if (st != SAQ_OK) return st;
    b.tile_start[0] = 0;
    b.tile_start[1] = (n + kBM - 1) / kBM * ex->npass;
    int *queue = nullptr;
    if (scratch_alloc((void **)&queue, 256, s) != cudaSuccess)
        return set_error(SAQ_ERR_OOM, "work counter allocation failed");
    st = SAQ_OK;
    if (cudaMemsetAsync(queue, 0, sizeof(int), s) != cudaSuccess)
        st = set_error(SAQ_ERR_CUDA, "work counter reset failed");
    if (st == SAQ_OK) st = launch_persistent<MODE>(b, m->tc.d_pad, queue, db, s);
    cudaFreeAsync(queue, s);
    return st;
}
}  // namespace

saq_status launch_project_tc_grouped(const ProjJob *jobs, int njobs, int *queue, cudaStream_t s) {
    if (njobs < 1 || njobs > kMaxGroups)
        return set_error(SAQ_ERR_INVALID, "1..%d models per grouped launch", kMaxGroups);
    int prec = -1;
    for (int i = 0; i < njobs; ++i) {
        const saq_model *m = jobs[i].m;
        if (m->dk == 0) continue;
        if (!tc_supported(m) || m->tc.precision != m->precision || m->precision == SAQ_PREC_FP32_SIMT)
            return set_error(SAQ_ERR_INVALID, "grouped projection needs tensor-core models");
        if (((uintptr_t)jobs[i].X & 15u) != 0) return set_error(SAQ_ERR_INVALID, "X not 16-byte aligned");
        if (m->kept.size() > 64) return set_error(SAQ_ERR_UNSUPPORTED, "more than 64 kept segments");
        if (prec >= 0 && m->tc.precision != prec)
            return set_error(SAQ_ERR_INVALID, "grouped projection needs one precision");
        prec = m->tc.precision;
    }
    switch (prec) {
        case -1: return SAQ_OK;
        case SAQ_PREC_FP32: return launch_grouped_mode<kSplit>(jobs, njobs, queue, s);
        case SAQ_PREC_BF16: return launch_grouped_mode<kBF16>(jobs, njobs, queue, s);
        case SAQ_PREC_FP8: return launch_grouped_mode<kFP8>(jobs, njobs, queue, s);
    }
    return set_error(SAQ_ERR_INVALID, "tensor-core operands not built");
}

saq_status tc_error_status(int code) {
    if (code == 0) return SAQ_OK;
    if (code == kErrRange)
        return set_error(SAQ_ERR_RANGE,
                         "tensor-core projection: an input row is not finite or lies outside the "
                         "range of the projection's operand format (|x - c| beyond about 8,000 "
                         "times the fitted per-coordinate rms for the FP32 split); the outputs of "
                         "that call are invalid");
    return set_error(SAQ_ERR_TIMEOUT, "tensor-core projection: a device wait timed out (role %d)",
                     code);
}

int *tc_error_word(const saq_model *m) {
    const TcExtra *ex = static_cast<const TcExtra *>(m->tc.extra);
    return ex ? ex->err : nullptr;
}

saq_status tc_check_error(const saq_model *m, cudaStream_t s) {
    const TcExtra *ex = static_cast<const TcExtra *>(m->tc.extra);
    if (!ex || !ex->err) return SAQ_OK;
    int h = 0;
    SAQ_CUDA_CHECK(cudaMemcpyAsync(&h, ex->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SAQ_CUDA_CHECK(cudaStreamSynchronize(s));
    if (h != 0) {
        cudaMemsetAsync(ex->err, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
        return tc_error_status(h);
    }
    return SAQ_OK;
}

}  // namespace saq

extern "C" saq_status saq_set_wait_limit(uint64_t ns) {
    saq::g_wait_ns.store(ns == 0 ? saq::kWaitNs : ns);
    return SAQ_OK;
}
