// storage.cuh -- how the (f_i, g_i) pairs are held in device memory.
//
// The state buffer holds plane 0 (the zeroth moments of the shifted sets) as FP32 pairs
// (padded to a multiple of 16 bytes for FP32 storage), followed by the shifted moving populations in the storage
// type:
//   STORE_F32   float2 (8 bytes per pair)
//   STORE_F16   __half2 (4 bytes), f scaled by 2^12 and g by 2^10 before rounding, so the
//               deviations sit in the normal FP16 range (|f - t w0| < 16, |g - t phi_ref| < 64)
//   STORE_BF16  __nv_bfloat162 (4 bytes), no scaling (BF16 has the FP32 exponent range)
// Each opposite pair of the velocity set is interleaved: pair plane k holds, per cell, the pair
// of population pair_first(k) then that of pair_second(k), one word of 16 bytes (FP32) or 8
// (16-bit). The Lax-Wendroff stencils of a population and its opposite read the same three
// cells, so one load serves both and the step issues half the loads and stores.
// All arithmetic is FP32 in every case. Plane 0 is 8 bytes whatever the storage: sum_i f_i - w0
// as FP32 and phi as the 32-bit integer phi * 2^30 (resolution 9.3e-10, range [-2, 2)). Each
// step adds to it the face fluxes of g rounded to that grid one face at a time; the two cells
// of a face round the same FP32 value, so the integers cancel in pairs and sum phi over the
// grid is conserved exactly, bit for bit, whatever precision the moving populations carry.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lattice.cuh"
#include "lbm_internal.h"

namespace lbm {

template <int S>
struct Store;

// Stored values are in storage units (scaled for FP16); kInvF / kInvG turn storage units into
// population units. load() applies them, store() applies kScaleF / kScaleG
// before rounding, store_raw() takes values already in storage units. The time step keeps the
// moving populations in storage units from load to store: propagation and collision are linear
// in them, the scales are powers of two (exact in FP32), so only the moments need rescaling and
// the results are the same bits as in population units.
//
// Raw pair access for the propagation: lo() and hi() take the pairs of a population and its
// opposite out of a loaded word, word() packs two for the store, cvt() converts a pair to
// FP32, sub_f(r, c) / sub_g(r, c) return (FP32 of r's f or g) - c with one rounding, sub2 both
// (for FP32 pairs one packed subtraction). For the
// 16-bit types these are the mixed-precision forms of sub (a 16-bit operand widened exactly to
// FP32, then subtracted), so a neighbour's pair is never converted on its own.
// a - b lane by lane in one packed FP32 instruction, each lane rounded as a scalar subtraction
__device__ __forceinline__ float2 fsub2_rn(float2 a, float2 b) {
    unsigned long long pa, pb, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(pa) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(pb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pa), "l"(pb));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(d));
    return o;
}

__device__ __forceinline__ void unpack16(unsigned int r, unsigned short& lo, unsigned short& hi) {
    asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(r));
}

template <>
struct Store<STORE_F32> {
    using T = float2;
    using Raw = float2;
    using Word = float4;  // the pairs of a population and its opposite
    static constexpr bool kUnsignedIndex = true;  // neighbour addresses from unsigned cell indices
    __device__ __forceinline__ static Raw lo(Word w) { return make_float2(w.x, w.y); }
    __device__ __forceinline__ static Raw hi(Word w) { return make_float2(w.z, w.w); }
    __device__ __forceinline__ static Word word(float fi, float gi, float fj, float gj) {
        return make_float4(fi, gi, fj, gj);
    }
    __device__ __forceinline__ static float2 cvt(Raw r) { return r; }
    __device__ __forceinline__ static float sub_f(Raw r, float c) { return __fsub_rn(r.x, c); }
    __device__ __forceinline__ static float sub_g(Raw r, float c) { return __fsub_rn(r.y, c); }
    __device__ __forceinline__ static float2 sub2(Raw r, float2 c) { return fsub2_rn(r, c); }
    static constexpr float kScaleF = 1.0f, kScaleG = 1.0f, kInvF = 1.0f, kInvG = 1.0f;
    __device__ __forceinline__ static float2 load(const T* p, const Params&) { return __ldg(p); }
    __device__ __forceinline__ static void store(T* p, float f, float g, const Params&) {
        __stcs(p, make_float2(f, g));
    }
    __device__ __forceinline__ static void store_raw(T* p, float f, float g) { __stcs(p, make_float2(f, g)); }
};

template <>
struct Store<STORE_F16> {
    using T = __half2;
    using Raw = unsigned int;
    using Word = uint2;
    static constexpr bool kUnsignedIndex = false;  // signed offsets: faster at the 96-register budget
    __device__ __forceinline__ static Raw lo(Word w) { return w.x; }
    __device__ __forceinline__ static Raw hi(Word w) { return w.y; }
    __device__ __forceinline__ static float2 cvt(Raw r) {
        return __half22float2(*reinterpret_cast<const __half2*>(&r));
    }
    __device__ __forceinline__ static float sub_f(Raw r, float c) {
        unsigned short lo, hi;
        unpack16(r, lo, hi);
        float d;
        asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(lo), "f"(c));
        return d;
    }
    __device__ __forceinline__ static float sub_g(Raw r, float c) {
        unsigned short lo, hi;
        unpack16(r, lo, hi);
        float d;
        asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(hi), "f"(c));
        return d;
    }
    __device__ __forceinline__ static float2 sub2(Raw r, float2 c) { return make_float2(sub_f(r, c.x), sub_g(r, c.y)); }
    static constexpr float kScaleF = 4096.0f, kScaleG = 1024.0f, kInvF = 1.0f / 4096.0f, kInvG = 1.0f / 1024.0f;
    __device__ __forceinline__ static float2 load(const T* p, const Params&) {
        const float2 v = __half22float2(__ldg(p));
        return make_float2(v.x * kInvF, v.y * kInvG);
    }
    __device__ __forceinline__ static void store(T* p, float f, float g, const Params&) {
        store_raw(p, f * kScaleF, g * kScaleG);
    }
    // the pair (f, g), already in storage units, rounded to its stored bits
    __device__ __forceinline__ static unsigned int pack_raw(float f, float g) {
        const __half2 h = __floats2half2_rn(f, g);
        return *reinterpret_cast<const unsigned int*>(&h);
    }
    __device__ __forceinline__ static void store_raw(T* p, float f, float g) {
        __stcs(reinterpret_cast<unsigned int*>(p), pack_raw(f, g));
    }
    __device__ __forceinline__ static Word word(float fi, float gi, float fj, float gj) {
        return make_uint2(pack_raw(fi, gi), pack_raw(fj, gj));
    }
};

template <>
struct Store<STORE_BF16> {
    using T = __nv_bfloat162;
    using Raw = unsigned int;
    using Word = uint2;
    static constexpr bool kUnsignedIndex = false;  // signed offsets: faster at the 96-register budget
    __device__ __forceinline__ static Raw lo(Word w) { return w.x; }
    __device__ __forceinline__ static Raw hi(Word w) { return w.y; }
    __device__ __forceinline__ static float2 cvt(Raw r) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r));
    }
    __device__ __forceinline__ static float sub_f(Raw r, float c) {
        unsigned short lo, hi;
        unpack16(r, lo, hi);
        float d;
        asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(lo), "f"(c));
        return d;
    }
    __device__ __forceinline__ static float sub_g(Raw r, float c) {
        unsigned short lo, hi;
        unpack16(r, lo, hi);
        float d;
        asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(hi), "f"(c));
        return d;
    }
    __device__ __forceinline__ static float2 sub2(Raw r, float2 c) { return make_float2(sub_f(r, c.x), sub_g(r, c.y)); }
    static constexpr float kScaleF = 1.0f, kScaleG = 1.0f, kInvF = 1.0f, kInvG = 1.0f;
    __device__ __forceinline__ static float2 load(const T* p, const Params&) { return __bfloat1622float2(__ldg(p)); }
    __device__ __forceinline__ static void store(T* p, float f, float g, const Params&) { store_raw(p, f, g); }
    __device__ __forceinline__ static unsigned int pack_raw(float f, float g) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f, g);
        return *reinterpret_cast<const unsigned int*>(&h);
    }
    __device__ __forceinline__ static void store_raw(T* p, float f, float g) {
        __stcs(reinterpret_cast<unsigned int*>(p), pack_raw(f, g));
    }
    __device__ __forceinline__ static Word word(float fi, float gi, float fj, float gj) {
        return make_uint2(pack_raw(fi, gi), pack_raw(fj, gj));
    }
};

// kInvG of a storage kind, for host code.
inline float storage_inv_g(int storage) { return storage == STORE_F16 ? Store<STORE_F16>::kInvG : 1.0f; }

// Fixed-point units of phi in plane 0.
constexpr double kPhiFx = 1073741824.0;  // 2^30
constexpr float kPhiFxInvF = 1.0f / 1073741824.0f;

// Plane 0 ((FP32, int32) pairs held as float2) and the moving planes of a state buffer.
__host__ __device__ __forceinline__ const float2* moment_plane(const void* state) {
    return static_cast<const float2*>(state);
}
__host__ __device__ __forceinline__ float2* moment_plane(void* state) { return static_cast<float2*>(state); }

// Bytes before the moving planes: plane 0, padded to a multiple of 16 for FP32 storage (its pair
// words are 16-byte loads). The 16-bit words need 8, which plane 0 always is; padding their offset
// too cost the 16-bit steps (held at 96 registers) spills and 2% of their rate (measured).
template <int S>
__host__ __device__ __forceinline__ size_t moving_offset(long long N) {
    if constexpr (S == STORE_F32) return ((size_t)N * sizeof(float2) + 15) & ~(size_t)15;
    else return (size_t)N * sizeof(float2);
}

// The pair plane of an opposite pair k (position of population i: pair_of, slot_of).
template <int Q>
__host__ __device__ constexpr int pair_of(int i) {
    for (int k = 0; k < Lat<Q>::kPairs; ++k)
        if (Lat<Q>::pair_first(k) == i || Lat<Q>::pair_second(k) == i) return k;
    return -1;
}
template <int Q>
__host__ __device__ constexpr int slot_of(int i) {
    return Lat<Q>::pair_second(pair_of<Q>(i)) == i ? 1 : 0;
}
template <int S>
__host__ __device__ __forceinline__ const typename Store<S>::Word* pair_plane(const void* state, long long N, int k) {
    return reinterpret_cast<const typename Store<S>::Word*>(static_cast<const char*>(state) + moving_offset<S>(N)) +
           (size_t)k * (size_t)N;
}
template <int S>
__host__ __device__ __forceinline__ typename Store<S>::Word* pair_plane(void* state, long long N, int k) {
    return reinterpret_cast<typename Store<S>::Word*>(static_cast<char*>(state) + moving_offset<S>(N)) + (size_t)k * (size_t)N;
}

// The stored pair of population i >= 1 at cell c.
template <int Q, int S>
__host__ __device__ __forceinline__ const typename Store<S>::T* pop_ptr(const void* state, long long N, int i, long long c) {
    return reinterpret_cast<const typename Store<S>::T*>(pair_plane<S>(state, N, pair_of<Q>(i)) + c) + slot_of<Q>(i);
}
template <int Q, int S>
__host__ __device__ __forceinline__ typename Store<S>::T* pop_ptr(void* state, long long N, int i, long long c) {
    return reinterpret_cast<typename Store<S>::T*>(pair_plane<S>(state, N, pair_of<Q>(i)) + c) + slot_of<Q>(i);
}

// Bytes of one state buffer.
inline size_t state_bytes(int Q, long long N, int storage) {
    if (storage == STORE_F32) return moving_offset<STORE_F32>(N) + (size_t)(Q - 1) * (size_t)N * sizeof(float2);
    return moving_offset<STORE_F16>(N) + (size_t)(Q - 1) * (size_t)N * 4;
}

}  // namespace lbm
