// k_caq1.cu -- quantize, adjust and pack one kept segment with one LANE per
// vector-segment (Sec. 3.1 Eq. find_nearest_code, Eq. adj-obj, Algorithm 1;
// Sec. 4.2 "quantize each segment separately").
//
// The 32 lanes of a warp run Algorithm 1 on 32 different vectors in lockstep
// over the coordinates of the segment: step j loads coordinate j of all 32
// vectors (one coalesced 128-byte line of the projected rows, stored
// interleaved by groups of 32 rows: O_i[(g * d_kept + col) * 32 + lane]) and
// reads their current codes from the warp's code store (packed 8 per batch in
// shared memory, k_caq1_sm, or one byte per coordinate in a global scratch
// with the rows' layout, k_caq1, when a block's codes do not fit), decides
// the lane's move against that lane's own state and applies it.  Each lane
// therefore executes the paper's sequential scan exactly, and an accepted
// move costs a predicated update instead of a serialising pass.
//
// Decision in closed form, without a division: with I = <u, o> > 0,
// S = |u|^2 and u = 2c - (2^B - 1), moving u_i by 2s (s = +-1) raises
// I^2 / S iff (I + 2 s o_i)^2 S > I^2 (S + 4 s u_i + 4), i.e. iff
//     s T I + o_i^2 S > I^2,   T = o_i S - u_i I.
// Only s = sign(T) can pass (the other side is smaller by 2|T|I), which is
// the convex-cone fact that at most one of +-Delta raises the cosine; the
// paper's -Delta trial after an accepted +Delta returns to the old point and
// is rejected.  The range check of c + s reads s*u < 2^B - 1.  A lane whose
// round made no move stops (its state no longer changes).  v_max comes from
// the projection (or a separate pass).  Every pass over the coordinates keeps
// kU loads in flight.  I and S are tracked in FP32 for the decisions; S is
// recounted exactly from the final codes while they are packed into
// bit-planes, during the last round (or, for a warp whose lanes all stop
// earlier, in a pass of its own).
#include <algorithm>
#include <atomic>

#include "saq_internal.h"

namespace saq {

namespace {

constexpr int kU = 8;  // loads in flight per lane in every pass
// the most dynamic shared memory a quantize block takes for its codes (at
// least three blocks of 256 threads per SM)
constexpr size_t kCaqSmemMax = 72 * 1024;
constexpr int kMaxSeg = 64;

struct Seg {
    int off, len, bits, words, fidx;
    long long code_off;
};
struct SegTable {
    Seg s[kMaxSeg];
    int order[kMaxSeg];  // segments by decreasing length: long work starts first
};
// One model's rows of a launch: its interleaved projected rows, byte-code
// scratch, v_max and outputs.
struct CaqGroup {
    const float *Oi;
    int64_t n;
    int dk, nseg, rounds, nf;
    uint8_t *cs;
    const float *vmax;
    uint8_t *codes;
    int64_t code_stride;
    float *factors;
    SegTable t;
};
// A launch over G models: global warp w belongs to the group g with
// warp_start[g] <= w < warp_start[g + 1] (ngroups <= G).
template <int G> struct CaqBatch {
    int ngroups;
    int64_t warp_start[G + 1];
    CaqGroup g[G];
};

// Where a lane keeps its vector-segment's codes during the adjustment.  Every
// access is by batches of kU = 8 coordinates starting at a multiple of 8,
// through a batch state held in registers:
//   load(j0, bt, n)      the batch of codes j0 .. j0 + n - 1 into bt
//   code(bt, k)          code j0 + k of the batch (0 past n)
//   move(bt, j0, k, c, sgn)  code j0 + k (now c) moves by one, up (sgn = 0)
//                        or down (sgn = 0x80000000), by an accepted move
//   flush(bt, j0)        after the batch's steps
//   write(j0, c, n)      store a batch's codes (the initial codes)
// GlobalCodes: one byte per coordinate in global memory, interleaved like
// the projected rows (byte j of the lane at j * 32), written at each move.
struct GlobalCodes {
    uint8_t *cp;
    static constexpr int kMinB = 1, kMaxB = 8;
    struct Batch {
        int c[kU];
    };
    __device__ __forceinline__ void load(int j0, Batch &bt, int n) const {
        if (n >= kU) {
#pragma unroll
            for (int k = 0; k < kU; ++k) bt.c[k] = (int)cp[(int64_t)(j0 + k) << 5];
        } else {
#pragma unroll
            for (int k = 0; k < kU; ++k) bt.c[k] = k < n ? (int)cp[(int64_t)(j0 + k) << 5] : 0;
        }
    }
    __device__ __forceinline__ int code(const Batch &bt, int k) const { return bt.c[k]; }
    __device__ __forceinline__ void write(int j0, const int (&c)[kU], int n) const {
#pragma unroll
        for (int k = 0; k < kU; ++k)
            if (k < n) cp[(int64_t)(j0 + k) << 5] = (uint8_t)c[k];
    }
    __device__ __forceinline__ void move(Batch &, int j0, int k, int c, uint32_t sgn) const {
        cp[(int64_t)(j0 + k) << 5] = (uint8_t)(sgn ? c - 1 : c + 1);
    }
    __device__ __forceinline__ void flush(Batch &, int) const {}
};
// SmemCodes<BITS>: packed in shared memory, BITS bits per code: 1 (B = 1),
// 2 (B = 2), 4 (B = 3, 4) or 8 (B = 5 .. 8).  A batch of 8 codes takes BITS
// bytes of the lane's byte stream, whose byte b is byte b % 4 of the lane's
// word b / 4, and word w of the lane sits at cw[w * 32] (the 32 lanes' words
// of one index are consecutive: no bank conflict).  A move adds +-1 to its
// code's field of the batch's value in a register (the range check keeps
// the field in [0, cmax]: no carry into the next field); the batch is stored
// back once, after its steps, as a byte, a half-word or one or two words, so
// that no other batch's codes are rewritten.
template <int BITS> struct SmemCodes {
    uint32_t *cw;
    static constexpr int kMinB = BITS == 1 ? 1 : BITS == 2 ? 2 : BITS == 4 ? 3 : 5, kMaxB = BITS;
    static constexpr int kWords = BITS >= 4 ? BITS / 4 : 1;  // registers per batch
    struct Batch {
        uint32_t w[kWords];
    };
    // the batch of coordinates j0 .. j0 + 7: its first word (BITS >= 4) or
    // its byte (BITS < 4)
    __device__ __forceinline__ uint32_t *word_of(int j0) const {
        return cw + (((j0 >> 3) * kWords) << 5);
    }
    __device__ __forceinline__ uint8_t *byte_of(int j0) const {
        const int bo = (j0 >> 3) * BITS;
        return reinterpret_cast<uint8_t *>(cw + ((bo >> 2) << 5)) + (bo & 3);
    }
    __device__ __forceinline__ uint32_t get(int j0) const {
        if constexpr (BITS == 1) return *byte_of(j0);
        else return *reinterpret_cast<const uint16_t *>(byte_of(j0));
    }
    __device__ __forceinline__ void set(int j0, uint32_t v) const {
        if constexpr (BITS == 1) *byte_of(j0) = (uint8_t)v;
        else *reinterpret_cast<uint16_t *>(byte_of(j0)) = (uint16_t)v;
    }
    __device__ __forceinline__ void store(int j0, const uint32_t (&w)[kWords]) const {
        if constexpr (BITS >= 4) {
#pragma unroll
            for (int i = 0; i < kWords; ++i) word_of(j0)[i << 5] = w[i];
        } else {
            set(j0, w[0]);
        }
    }
    __device__ __forceinline__ void load(int j0, Batch &bt, int) const {
        if constexpr (BITS >= 4) {
#pragma unroll
            for (int i = 0; i < kWords; ++i) bt.w[i] = word_of(j0)[i << 5];
        } else {
            bt.w[0] = get(j0);
        }
    }
    __device__ __forceinline__ int code(const Batch &bt, int k) const {
        return (int)((bt.w[k * BITS / 32] >> ((k * BITS) & 31)) & ((1u << BITS) - 1u));
    }
    __device__ __forceinline__ void write(int j0, const int (&c)[kU], int n) const {
        uint32_t w[kWords];
#pragma unroll
        for (int i = 0; i < kWords; ++i) w[i] = 0u;
#pragma unroll
        for (int k = 0; k < kU; ++k)
            if (k < n) w[k * BITS / 32] |= (uint32_t)c[k] << ((k * BITS) & 31);
        store(j0, w);
    }
    __device__ __forceinline__ void move(Batch &bt, int, int k, int, uint32_t sgn) const {
        const uint32_t one = 1u << ((k * BITS) & 31);
        bt.w[k * BITS / 32] += sgn ? 0u - one : one;
    }
    __device__ __forceinline__ void flush(Batch &bt, int j0) const { store(j0, bt.w); }
};

// Bit-planes of one lane's segment from its codes (most significant first,
// 64-bit words); returns |u|^2 of the codes, exactly.
template <int B, class CS>
__device__ __forceinline__ int pack_segment(const CS &cs, int len, bool valid,
                                            uint64_t *cout, int words) {
    constexpr int cmax = (1 << B) - 1;
    uint64_t w[B];
#pragma unroll
    for (int p = 0; p < B; ++p) w[p] = 0ull;
    int S = 0;
    for (int j0 = 0; j0 < len; j0 += kU) {
        typename CS::Batch bt;
        cs.load(j0, bt, len - j0);
        int c[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) c[k] = cs.code(bt, k);
        // plane p of the kU codes as the bits of one byte (past the end: 0)
#pragma unroll
        for (int p = 0; p < B; ++p) {
            uint32_t b = 0;
#pragma unroll
            for (int k = 0; k < kU; ++k) b |= (uint32_t)((c[k] >> (B - 1 - p)) & 1) << k;
            w[p] |= (uint64_t)b << (j0 & 63);
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int u = 2 * c[k] - cmax;
            S += j0 + k < len ? u * u : 0;  // a code past the end reads 0, not a code
        }
        if (((j0 + kU) & 63) == 0 || j0 + kU >= len) {
            if (valid) {
#pragma unroll
                for (int p = 0; p < B; ++p) cout[p * words + (j0 >> 6)] = w[p];
            }
#pragma unroll
            for (int p = 0; p < B; ++p) w[p] = 0ull;
        }
    }
    return S;
}

// The adjustment state of one lane's vector-segment.  A lane that is done
// (no move in its last round, or nothing to adjust) holds I2 = +inf, which
// no gain exceeds.
struct LaneState {
    float I, S, I2;
};

// One coordinate of Algorithm 1 for one lane: returns the coordinate's code
// after the step and sets `accepted` if it moved.  u = 2c - cmax is formed
// as a float without a conversion: the bits 0x4B400000 + (2c - cmax) are the
// float 1.5 * 2^23 + (2c - cmax) exactly (unit spacing there), ubias =
// 0x4B400000 - cmax; s = sign(T) (+ for T = +0); s*u < cmax is the range
// check of c + s.
__device__ __forceinline__ bool caq_move(LaneState &L, float x, int c, int ubias, float cmaxf,
                                         uint32_t &sgn) {
    const float u = __int_as_float(ubias + 2 * c) - 12582912.f;
    const float xS = x * L.S;
    const float T = fmaf(-u, L.I, xS);
    sgn = __float_as_uint(T) & 0x80000000u;
    const float su = __uint_as_float(__float_as_uint(u) ^ sgn);
    if (su < cmaxf && fmaf(fabsf(T), L.I, x * xS) > L.I2) {
        L.I = fmaf(__uint_as_float(0x40000000u | sgn), x, L.I);
        L.S = fmaf(4.f, su, L.S + 4.f);
        L.I2 = L.I * L.I;
        return true;
    }
    return false;
}
__device__ __forceinline__ int caq_step(LaneState &L, float x, int c, int ubias, float cmaxf,
                                        bool &accepted) {
    uint32_t sgn;
    if (caq_move(L, x, c, ubias, cmaxf, sgn)) {
        c = sgn ? c - 1 : c + 1;
        accepted = true;
    }
    return c;
}

// One round of Algorithm 1 over the lane's segment: coordinates j0 + U ..
// j0 + 2U - 1 are loaded before j0 .. j0 + U - 1 are processed (a code is only
// written at its own step, so the prefetched codes are current).  With
// PACK_B = B > 0 the round is the last one: a coordinate's code is final once
// its own step is done, so the bit-planes (most significant first, 64-bit
// words) and the exact |u|^2, which the function returns, are built as the
// round goes.
template <int PACK_B, class CS>
__device__ __forceinline__ int run_round(LaneState &L, const float *op, const CS &cs, int len,
                                         int cmax, bool &moved, bool valid, uint64_t *cout,
                                         int words) {
    const int ubias = 0x4B400000 - cmax;
    const float cmaxf = (float)cmax;
    const int lenU = len & ~(kU - 1);  // coordinates in whole batches
    constexpr int NW = PACK_B > 0 ? PACK_B : 1;
    uint64_t w[NW];
#pragma unroll
    for (int p = 0; p < NW; ++p) w[p] = 0ull;
    int Si = 0;
    typename CS::Batch bb, bn;  // the current and the next batch's code state
    // the step of coordinate j0 + k (its code read from the batch state just
    // before the step: earlier moves of the batch touch only other codes);
    // returns the code after the step when the round packs (else unused)
    auto step = [&](float x, int j0, int k) {
        const int c = cs.code(bb, k);
        uint32_t sgn;
        const bool acc = caq_move(L, x, c, ubias, cmaxf, sgn);
        if (acc) {
            cs.move(bb, j0, k, c, sgn);
            moved = true;
        }
        return PACK_B > 0 && acc ? (sgn ? c - 1 : c + 1) : c;
    };
    // the final codes cf[0 .. count) of the batch at j0 into the planes
    auto pack = [&](const int (&cf)[kU], int j0, int count) {
        if (PACK_B == 0) return;
#pragma unroll
        for (int p = 0; p < NW; ++p) {
            uint32_t b = 0;
#pragma unroll
            for (int k = 0; k < kU; ++k)
                if (k < count) b |= (uint32_t)((cf[k] >> (NW - 1 - p)) & 1) << k;
            w[p] |= (uint64_t)b << (j0 & 63);
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int u = 2 * cf[k] - cmax;
            if (k < count) Si += u * u;
        }
        if (((j0 + kU) & 63) == 0 || j0 + count >= len) {
            if (valid) {
#pragma unroll
                for (int p = 0; p < NW; ++p) cout[p * words + (j0 >> 6)] = w[p];
            }
#pragma unroll
            for (int p = 0; p < NW; ++p) w[p] = 0ull;
        }
    };
    float xb[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) xb[k] = k < len ? __ldg(op + ((int64_t)k << 5)) : 0.f;
    cs.load(0, bb, len);
    for (int j0 = 0; j0 < lenU; j0 += kU) {
        float xn[kU];
        if (j0 + 2 * kU <= len) {  // the next batch lies inside the segment
#pragma unroll
            for (int k = 0; k < kU; ++k) xn[k] = __ldg(op + ((int64_t)(j0 + kU + k) << 5));
        } else {
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                const int jn = j0 + kU + k;
                xn[k] = jn < len ? __ldg(op + ((int64_t)jn << 5)) : 0.f;
            }
        }
        // the next batch's codes (a code is written at its own step, and a
        // batch is stored back after its steps: the next one is current)
        if (j0 + kU < len) cs.load(j0 + kU, bn, len - j0 - kU);
        int cf[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) cf[k] = step(xb[k], j0, k);
        cs.flush(bb, j0);
        pack(cf, j0, kU);
        bb = bn;
#pragma unroll
        for (int k = 0; k < kU; ++k) xb[k] = xn[k];
    }
    // the last, partial batch
    if (lenU < len) {
        int cf[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) cf[k] = lenU + k < len ? step(xb[k], lenU, k) : 0;
        cs.flush(bb, lenU);
        pack(cf, lenU, len - lenU);
    }
    return Si;
}

// The last round (which packs as it goes) and the separate packing pass for
// B bits, instantiated only for the bit widths the code store holds.
template <int B, class CS>
__device__ __forceinline__ int last_round(LaneState &L, const float *op, const CS &cs, int len,
                                          int cmax, bool &moved, bool valid, uint64_t *cout,
                                          int words) {
    if constexpr (B >= CS::kMinB && B <= CS::kMaxB)
        return run_round<B, CS>(L, op, cs, len, cmax, moved, valid, cout, words);
    else
        return 0;
}
template <int B, class CS>
__device__ __forceinline__ int pack_only(const CS &cs, int len, bool valid, uint64_t *cout,
                                         int words) {
    if constexpr (B >= CS::kMinB && B <= CS::kMaxB)
        return pack_segment<B, CS>(cs, len, valid, cout, words);
    else
        return 0;
}

// Algorithm 1 on one lane's vector-segment with its codes in store cs:
// initial codes, the rounds, the packing and the two factors.
template <class CS>
__device__ __forceinline__ void caq_segment(const CS &cs, const float *op, int len, int B,
                                            int words, bool valid, float vmax, int rounds,
                                            uint64_t *cout, float *fo) {
    const int cmax = (1 << B) - 1;
    const bool live = valid && vmax > 0.f;
    // initial codes, Eq. find_nearest_code: c = floor((o + v_max) / Delta),
    // Delta = 2 v_max / 2^B; with I = <u, o>, S = |u|^2 and |o|^2
    // (in FP32: the code c as a float, clamped, the integer from the bits of
    // c + 2^23; |u|^2 is summed in FP32 for the decisions and recounted
    // exactly while packing).  Every lane of the last group of 32 rows reads
    // rows the buffer holds; a lane past n keeps codes 0.
    const float inv_delta = live ? (float)(1 << (B - 1)) / vmax : 0.f;
    const float off_c = vmax * inv_delta;  // (o + v_max) / Delta = o / Delta + off_c
    const float cmaxf = (float)cmax;
    float I = 0.f, n2 = 0.f, S = 0.f;
    auto init = [&](float x) {
        const float cf = fminf(fmaxf(floorf(fmaf(x, inv_delta, off_c)), 0.f), cmaxf);
        const float u = fmaf(2.f, cf, -cmaxf);
        I = fmaf(u, x, I);
        n2 = fmaf(x, x, n2);
        S = fmaf(u, u, S);
        return (int)(__float_as_uint(cf + 8388608.f) & 0xFFu);
    };
    const int lenU = len & ~(kU - 1);  // coordinates in whole batches
    for (int j0 = 0; j0 < lenU; j0 += kU) {
        float x[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) x[k] = __ldg(op + ((int64_t)(j0 + k) << 5));
        int c[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) c[k] = init(live ? x[k] : 0.f);
        cs.write(j0, c, kU);
    }
    if (lenU < len) {
        int c[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k)
            c[k] = lenU + k < len ? init(live ? __ldg(op + ((int64_t)(lenU + k) << 5)) : 0.f) : 0;
        cs.write(lenU, c, len - lenU);
    }
    LaneState L{I, S, live ? I * I : __int_as_float(0x7f800000)};
    int Si = -1;  // |u|^2 of the final codes, exactly, once they are packed
    for (int r = 0; r < rounds; ++r) {
        if (!__any_sync(0xffffffffu, L.I2 != __int_as_float(0x7f800000))) break;
        bool moved = false;
        if (r == rounds - 1) {  // the last round packs as it goes
            switch (B) {  // uniform per warp
                case 1: Si = last_round<1, CS>(L, op, cs, len, cmax, moved, valid, cout, words); break;
                case 2: Si = last_round<2, CS>(L, op, cs, len, cmax, moved, valid, cout, words); break;
                case 3: Si = last_round<3, CS>(L, op, cs, len, cmax, moved, valid, cout, words); break;
                case 4: Si = last_round<4, CS>(L, op, cs, len, cmax, moved, valid, cout, words); break;
                case 5: Si = last_round<5, CS>(L, op, cs, len, cmax, moved, valid, cout, words); break;
                case 6: Si = last_round<6, CS>(L, op, cs, len, cmax, moved, valid, cout, words); break;
                case 7: Si = last_round<7, CS>(L, op, cs, len, cmax, moved, valid, cout, words); break;
                default: Si = last_round<8, CS>(L, op, cs, len, cmax, moved, valid, cout, words); break;
            }
            break;
        }
        run_round<0, CS>(L, op, cs, len, cmax, moved, valid, cout, words);
        if (!moved) L.I2 = __int_as_float(0x7f800000);
    }
    I = L.I;
    // every lane done before the last round (or no rounds): pack from the codes
    if (Si < 0) {
        switch (B) {  // uniform per warp
            case 1: Si = pack_only<1, CS>(cs, len, valid, cout, words); break;
            case 2: Si = pack_only<2, CS>(cs, len, valid, cout, words); break;
            case 3: Si = pack_only<3, CS>(cs, len, valid, cout, words); break;
            case 4: Si = pack_only<4, CS>(cs, len, valid, cout, words); break;
            case 5: Si = pack_only<5, CS>(cs, len, valid, cout, words); break;
            case 6: Si = pack_only<6, CS>(cs, len, valid, cout, words); break;
            case 7: Si = pack_only<7, CS>(cs, len, valid, cout, words); break;
            default: Si = pack_only<8, CS>(cs, len, valid, cout, words); break;
        }
    }
    if (valid) {
        if (live) {
            const float nrm = sqrtf(n2);
            fo[0] = nrm;
            fo[1] = I / (sqrtf((float)Si) * nrm);
        } else {
            // all-zero segment (the paper is silent): codes 0, |o| = 0, cos = 1
            fo[0] = 0.f;
            fo[1] = 1.f;
        }
    }
}

// The work of warp w of one model's launch: one warp per (kept segment,
// group of 32 rows).  SMEM_CODES: the codes live in the warp's region of
// the block's shared memory (words_per_lane 32-bit words per lane), else in
// the byte scratch cs.
template <bool SMEM_CODES>
__device__ __forceinline__ void caq1_warp(int64_t w, const float *__restrict__ Oi, int64_t n,
                                          int dk, int nseg, const SegTable &t, int rounds,
                                          uint8_t *__restrict__ cs,
                                          const float *__restrict__ vmax_arr,
                                          uint8_t *__restrict__ codes, int64_t code_stride,
                                          float *__restrict__ factors, int nf,
                                          uint32_t *smem_codes, int words_per_lane) {
    const int lane = threadIdx.x & 31;
    const int64_t groups = (n + 31) / 32;
    const int si = t.order[w / groups];
    const Seg sg = t.s[si];
    const int64_t g = w % groups;
    const int off = sg.off, len = sg.len, B = sg.bits, words = sg.words, fidx = sg.fidx;
    const long long code_off = sg.code_off;
    const int64_t v = g * 32 + lane;
    const bool valid = v < n;
    const float *op = Oi + ((g * dk + off) << 5) + lane;
    // v_max of the lane's vector-segment, recorded by the projection
    const float vmax = valid ? __ldg(vmax_arr + ((g * nseg + si) << 5) + lane) : 0.f;
    uint64_t *cout = reinterpret_cast<uint64_t *>(codes + v * code_stride + code_off);
    float *fo = factors + v * nf + fidx;
    if constexpr (SMEM_CODES) {
        uint32_t *cw = smem_codes + (threadIdx.x >> 5) * (words_per_lane << 5) + lane;
        if (B == 1)  // uniform per warp
            caq_segment(SmemCodes<1>{cw}, op, len, B, words, valid, vmax, rounds, cout, fo);
        else if (B == 2)
            caq_segment(SmemCodes<2>{cw}, op, len, B, words, valid, vmax, rounds, cout, fo);
        else if (B <= 4)
            caq_segment(SmemCodes<4>{cw}, op, len, B, words, valid, vmax, rounds, cout, fo);
        else
            caq_segment(SmemCodes<8>{cw}, op, len, B, words, valid, vmax, rounds, cout, fo);
    } else {
        caq_segment(GlobalCodes{cs + ((g * dk + off) << 5) + lane}, op, len, B, words, valid, vmax,
                    rounds, cout, fo);
    }
}

// All kept segments of a chunk in one launch.  Four blocks of 256 threads
// per SM (64 registers): the packing round spills a little, which costs less
// than the lower occupancy of an uncapped build.
__global__ void __launch_bounds__(256, 4)
k_caq1(const float *__restrict__ Oi, int64_t n, int dk, int nseg, const SegTable t, int rounds,
       uint8_t *__restrict__ cs, const float *__restrict__ vmax_arr,
       uint8_t *__restrict__ codes, int64_t code_stride, float *__restrict__ factors, int nf) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (n + 31) / 32 * nseg) return;  // uniform per warp
    caq1_warp<false>(w, Oi, n, dk, nseg, t, rounds, cs, vmax_arr, codes, code_stride, factors, nf,
                     nullptr, 0);
}

// The same with every warp's codes in shared memory (words_per_lane 32-bit
// words per lane: 4-bit codes for B <= 4, bytes above): the adjustment
// rounds then read only the projected rows from global memory.
__global__ void __launch_bounds__(256, 4)
k_caq1_sm(const float *__restrict__ Oi, int64_t n, int dk, int nseg, const SegTable t, int rounds,
          const float *__restrict__ vmax_arr, uint8_t *__restrict__ codes, int64_t code_stride,
          float *__restrict__ factors, int nf, int words_per_lane) {
    extern __shared__ uint32_t smem_codes[];
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (n + 31) / 32 * nseg) return;  // uniform per warp
    caq1_warp<true>(w, Oi, n, dk, nseg, t, rounds, nullptr, vmax_arr, codes, code_stride, factors,
                    nf, smem_codes, words_per_lane);
}

// The rows of up to kMaxGroups models (a batch of several collections) in
// one launch: global warp w belongs to the group g with warp_start[g] <= w <
// warp_start[g + 1].
// A persistent warp of a grouped launch: it takes work items (global warp
// indices of the batch) from the device counter `queue` until none is left.
template <bool SMEM_CODES>
__device__ __forceinline__ void caq1_grouped_warp(const CaqBatch<kMaxGroups> &batch, int *queue,
                                                  uint32_t *smem_codes, int words_per_lane) {
    const int64_t total = batch.warp_start[batch.ngroups];
    for (;;) {
        int wi = 0;
        if ((threadIdx.x & 31) == 0) wi = atomicAdd(queue, 1);
        const int64_t wg = __shfl_sync(0xffffffffu, wi, 0);
        if (wg >= total) break;  // uniform per warp
        int gi = 0;
        while (gi + 1 < batch.ngroups && wg >= batch.warp_start[gi + 1]) ++gi;
        const CaqGroup &P = batch.g[gi];
        caq1_warp<SMEM_CODES>(wg - batch.warp_start[gi], P.Oi, P.n, P.dk, P.nseg, P.t, P.rounds,
                              P.cs, P.vmax, P.codes, P.code_stride, P.factors, P.nf, smem_codes,
                              words_per_lane);
    }
}
__global__ void __launch_bounds__(256, 4)
k_caq1_grouped(const __grid_constant__ CaqBatch<kMaxGroups> batch, int *queue) {
    caq1_grouped_warp<false>(batch, queue, nullptr, 0);
}
// The same with the codes in shared memory (words_per_lane: the largest
// over the groups' segments).
__global__ void __launch_bounds__(256, 4)
k_caq1_grouped_sm(const __grid_constant__ CaqBatch<kMaxGroups> batch, int *queue,
                  int words_per_lane) {
    extern __shared__ uint32_t smem_codes[];
    caq1_grouped_warp<true>(batch, queue, smem_codes, words_per_lane);
}

// The instruction ceiling of the adjustment: caq_step on coordinates held in
// registers (no loads or stores), kU per lane, a sign flip per step keeping
// moves happening; one block of 128 threads per 4 warps of occupancy.
__global__ void __launch_bounds__(128) k_step_ceiling(int iters, int cmax, float *out) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    float x[kU];
    int c[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
        x[k] = (float)((tid * 7 + k * 13) % 31) * 0.03f - 0.45f;
        c[k] = (tid + k) % (cmax + 1);
    }
    LaneState L{10.f, 200.f, 100.f};
    const int ubias = 0x4B400000 - cmax;
    const float cmaxf = (float)cmax;
    int moves = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            bool accepted = false;
            c[k] = caq_step(L, x[k], c[k], ubias, cmaxf, accepted);
            moves += accepted ? 1 : 0;
            x[k] = -x[k];
        }
    }
    out[tid] = L.I + L.S + (float)moves + (float)c[0];
}

// v_max of every (row, kept segment) of interleaved rows: one warp per (group
// of 32 rows, kept segment), lane = row.
__global__ void __launch_bounds__(256)
k_seg_vmax(const float *__restrict__ Oi, int64_t n, int dk, const SegCols sc,
           float *__restrict__ vmax) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t groups = (n + 31) / 32;
    if (w >= groups * sc.nk) return;
    const int64_t g = w / sc.nk;
    const int s = (int)(w % sc.nk);
    const int c0 = s == 0 ? 0 : sc.end[s - 1], c1 = sc.end[s];
    const bool valid = g * 32 + lane < n;
    float mx = 0.f;
    for (int c = c0; c < c1; ++c)
        mx = fmaxf(mx, valid ? fabsf(__ldg(Oi + ((g * dk + c) << 5) + lane)) : 0.f);
    vmax[((g * sc.nk + s) << 5) + lane] = mx;
}

// Row-major O (n x dk, ldo) -> interleaved O_i (groups of 32 rows).
__global__ void k_interleave(const float *__restrict__ O, int64_t ldo, int64_t n, int dk,
                             float *__restrict__ Oi) {
    __shared__ float tile[32][33];
    const int64_t g = blockIdx.y;
    const int c0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int rr = ty; rr < 32; rr += 8) {
        const int64_t row = g * 32 + rr;
        const int col = c0 + tx;
        tile[rr][tx] = (row < n && col < dk) ? O[row * ldo + col] : 0.f;
    }
    __syncthreads();
    for (int cc = ty; cc < 32; cc += 8) {
        const int col = c0 + cc;
        if (col < dk) Oi[((g * dk + col) << 5) + tx] = tile[tx][cc];
    }
}

}  // namespace

namespace {

saq_status make_group(const CaqJob &j, CaqGroup *g) {
    const saq_model *m = j.m;
    const int nk = (int)m->kept.size();
    if (nk > kMaxSeg) return set_error(SAQ_ERR_UNSUPPORTED, "more than %d kept segments", kMaxSeg);
    SegTable &t = g->t;
    for (int i = 0; i < nk; ++i) {
        const KeptSeg &k = m->kept[(size_t)i];
        if (k.bits < 1 || k.bits > 8)
            return set_error(SAQ_ERR_INVALID, "segment bits %d outside 1..8", k.bits);
        t.s[i] = Seg{k.off, k.len, k.bits, k.words, k.fidx, (long long)k.code_off};
        t.order[i] = i;
    }
    std::stable_sort(t.order, t.order + nk, [&](int a, int b) { return t.s[a].len > t.s[b].len; });
    g->Oi = j.Oi;
    g->n = j.n;
    g->dk = m->dk;
    g->nseg = nk;
    g->rounds = m->rounds;
    g->nf = m->nf;
    g->cs = j.cs;
    g->vmax = j.vmax;
    g->codes = j.codes;
    g->code_stride = (int64_t)m->code_bytes;
    g->factors = j.factors;
    return SAQ_OK;
}

// 32-bit words per lane of the shared-memory code store for model m: its
// largest segment's, at 1, 2, 4 or 8 bits per code (B = 1, 2, 3-4, 5-8),
// a batch of 8 codes in that many bytes.
int words_per_lane(const saq_model *m) {
    int wpl = 0;
    for (const KeptSeg &k : m->kept) {
        const int width = k.bits <= 1 ? 1 : k.bits == 2 ? 2 : k.bits <= 4 ? 4 : 8;
        wpl = std::max(wpl, ((k.len + 7) / 8 * width + 3) / 4);
    }
    return wpl;
}

// Shared memory of a block of 8 warps for wpl words per lane; the codes go
// to shared memory when it is at most kCaqSmemMax (at least 3 blocks per SM).
size_t caq_smem_bytes(int wpl) { return (size_t)wpl * 32 * 4 * 8; }

// Sets the kernel's shared-memory attributes once per device (`done`: one
// bit per device ordinal, devices 0..63; a larger ordinal sets them at
// every launch).
template <class K> saq_status prepare_smem_kernel(K *kernel, std::atomic<uint64_t> &done) {
    int dev = 0;
    SAQ_CUDA_CHECK(cudaGetDevice(&dev));
    const uint64_t bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return SAQ_OK;
    SAQ_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kCaqSmemMax));
    // all of the unified L1 / shared storage as shared memory: four blocks
    // of 56 KB fit (the d = 960 plan's longest segment)
    SAQ_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        100));
    done.fetch_or(bit, std::memory_order_release);
    return SAQ_OK;
}
std::atomic<uint64_t> g_caq1_sm_ready{0}, g_caq1_grouped_sm_ready{0};

}  // namespace

saq_status launch_caq1(const saq_model *m, const float *Oi, int64_t n, uint8_t *cs,
                       const float *vmax, uint8_t *codes, float *factors, cudaStream_t s) {
    if (n <= 0 || m->kept.empty()) return SAQ_OK;
    CaqGroup g;
    saq_status st = make_group(CaqJob{m, Oi, n, cs, vmax, codes, factors}, &g);
    if (st != SAQ_OK) return st;
    const int64_t warps = (n + 31) / 32 * g.nseg;
    const int64_t blocks = (warps + 7) / 8;
    // codes in shared memory when they fit, else in the global byte scratch
    const int wpl = words_per_lane(m);
    const size_t smem = caq_smem_bytes(wpl);
    if (smem <= kCaqSmemMax) {
        st = prepare_smem_kernel(k_caq1_sm, g_caq1_sm_ready);
        if (st != SAQ_OK) return st;
    }
    {
        LaunchTimer lt_(kKindQuantize, s);
        if (smem <= kCaqSmemMax) {
            k_caq1_sm<<<(unsigned)blocks, 256, smem, s>>>(Oi, n, g.dk, g.nseg, g.t, g.rounds, vmax,
                                                          codes, g.code_stride, factors, g.nf, wpl);
        } else {
            k_caq1<<<(unsigned)blocks, 256, 0, s>>>(Oi, n, g.dk, g.nseg, g.t, g.rounds, cs, vmax,
                                                    codes, g.code_stride, factors, g.nf);
        }
    }
    note_launches();
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

saq_status launch_caq1_grouped(const CaqJob *jobs, int njobs, int *queue, cudaStream_t s) {
    if (njobs < 1 || njobs > kMaxGroups)
        return set_error(SAQ_ERR_INVALID, "1..%d models per grouped launch", kMaxGroups);
    CaqBatch<kMaxGroups> b;
    b.ngroups = 0;
    b.warp_start[0] = 0;
    int wpl = 0;
    for (int i = 0; i < njobs; ++i) {
        if (jobs[i].n <= 0 || jobs[i].m->kept.empty()) continue;
        wpl = std::max(wpl, words_per_lane(jobs[i].m));
        saq_status st = make_group(jobs[i], &b.g[b.ngroups]);
        if (st != SAQ_OK) return st;
        b.warp_start[b.ngroups + 1] =
            b.warp_start[b.ngroups] + (jobs[i].n + 31) / 32 * (int64_t)b.g[b.ngroups].nseg;
        ++b.ngroups;
    }
    if (b.ngroups == 0) return SAQ_OK;
    if (b.warp_start[b.ngroups] > 0x7FFFFFFF)
        return set_error(SAQ_ERR_UNSUPPORTED, "too many rows in one call");
    const int64_t blocks = (b.warp_start[b.ngroups] + 7) / 8;
    const size_t smem = caq_smem_bytes(wpl);
    const bool sm_codes = smem <= kCaqSmemMax;
    if (sm_codes) {
        saq_status st = prepare_smem_kernel(k_caq1_grouped_sm, g_caq1_grouped_sm_ready);
        if (st != SAQ_OK) return st;
    }
    // persistent: as many blocks as stay resident at once (at most the work)
    int dev = 0, sms = 0, per_sm = 0;
    SAQ_CUDA_CHECK(cudaGetDevice(&dev));
    SAQ_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (sm_codes)
        SAQ_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_caq1_grouped_sm, 256,
                                                                     smem));
    else
        SAQ_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_caq1_grouped, 256, 0));
    const int64_t grid = std::min<int64_t>(blocks, (int64_t)std::max(1, sms * per_sm));
    {
        LaunchTimer lt_(kKindQuantize, s);
        if (sm_codes)
            k_caq1_grouped_sm<<<(unsigned)grid, 256, smem, s>>>(b, queue, wpl);
        else
            k_caq1_grouped<<<(unsigned)grid, 256, 0, s>>>(b, queue);
    }
    note_launches();
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

saq_status step_ceiling(int warps_per_sm, int bits, double *lane_steps_per_s) {
    int dev = 0, sms = 0;
    SAQ_CUDA_CHECK(cudaGetDevice(&dev));
    SAQ_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * (warps_per_sm / 4);
    const int iters = 2000;
    float *out = nullptr;
    SAQ_CUDA_CHECK(scratch_alloc((void **)&out, sizeof(float) * (size_t)blocks * 128, 0));
    cudaEvent_t a = nullptr, b = nullptr;
    saq_status st = SAQ_OK;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        st = set_error(SAQ_ERR_CUDA, "event creation failed");
    } else {
        const int cmax = (1 << bits) - 1;
        k_step_ceiling<<<blocks, 128>>>(iters / 4, cmax, out);  // warm-up
        cudaEventRecord(a, 0);
        k_step_ceiling<<<blocks, 128>>>(iters, cmax, out);
        cudaEventRecord(b, 0);
        note_launches(2);
        float ms = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess || ms <= 0.f)
            st = set_error(SAQ_ERR_CUDA, "step-ceiling measurement failed");
        else
            *lane_steps_per_s = (double)blocks * 128.0 * iters * kU / (ms * 1e-3);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFreeAsync(out, 0);
    cudaStreamSynchronize(0);
    return st;
}

saq_status launch_seg_vmax(const saq_model *m, const float *Oi, int64_t n, float *vmax,
                           cudaStream_t s) {
    const SegCols sc = seg_cols(m);
    if (n <= 0 || sc.nk == 0) return SAQ_OK;
    const int64_t warps = (n + 31) / 32 * sc.nk;
    {
        LaunchTimer lt_(kKindOther, s);
        k_seg_vmax<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(Oi, n, m->dk, sc, vmax);
    }
    note_launches();
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

saq_status launch_interleave(const float *O, int64_t ldo, int64_t n, int dk, float *Oi,
                             cudaStream_t s) {
    if (n <= 0 || dk <= 0) return SAQ_OK;
    const int64_t groups = (n + 31) / 32;
    dim3 grid((unsigned)((dk + 31) / 32), (unsigned)groups);
    if (groups > 65535) {
        // split along groups to respect the grid's y limit
        for (int64_t g0 = 0; g0 < groups; g0 += 65535) {
            const int64_t gn = std::min<int64_t>(65535, groups - g0);
            dim3 gg((unsigned)((dk + 31) / 32), (unsigned)gn);
            {
                LaunchTimer lt_(kKindOther, s);
                k_interleave<<<gg, dim3(32, 8), 0, s>>>(O + g0 * 32 * ldo, ldo, n - g0 * 32, dk,
                                                        Oi + g0 * 32 * (int64_t)dk);
            }
            note_launches();
        }
    } else {
        {
            LaunchTimer lt_(kKindOther, s);
            k_interleave<<<grid, dim3(32, 8), 0, s>>>(O, ldo, n, dk, Oi);
        }
        note_launches();
    }
    SAQ_CUDA_CHECK(cudaGetLastError());
    return SAQ_OK;
}

}  // namespace saq
