// Shared pieces of the peak-detection kernels (Sec. 4.4): the total-order key
// of a map cell, the wrap-around index, and the block-wide radix selection of
// the largest keys.
#pragma once

#include "ft_internal.cuh"

typedef unsigned long long u64;

__device__ __forceinline__ u64 peak_key(float v, unsigned lin) {
    return ((u64)__float_as_uint(v) << 32) | (u64)(0xFFFFFFFFu - lin);
}

__device__ __forceinline__ int wrap_into(int a, int n) {
    if (a < 0) a += n;
    if (a >= n) a %= n;
    return a;
}

// Bitonic sort, descending, of n (power of two) keys in shared memory.
static __device__ void bitonic_desc(u64* v, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool desc = (i & k) == 0;
                    const u64 x = v[i], y = v[ixj];
                    if (desc ? (x < y) : (x > y)) {
                        v[i] = y;
                        v[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

struct SelState {
    unsigned hist[256];
    u64 prefix, mask;
    int remaining;
    int done;
    int count;
};

// Marks the top K non-zero keys key_of(0 .. n-1) (distinct unless zero): on
// return every key k != 0 with (k & st.mask) >= st.prefix is selected and there
// are exactly min(K, #non-zero keys) of them.  Called by the whole block.
template <typename KeyOf>
static __device__ void cta_select_by(int n, int K, SelState& st, KeyOf key_of) {
    if (threadIdx.x == 0) {
        st.prefix = 0ull;
        st.mask = 0ull;
        st.remaining = K;
        st.done = 0;
    }
    __syncthreads();
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) st.hist[i] = 0u;
        __syncthreads();
        const u64 pf = st.prefix, mk = st.mask;
        for (int i0 = threadIdx.x & ~31; i0 < n; i0 += blockDim.x) {
            // keys share their leading digits, so lanes with equal digits add once
            const int i = i0 + (threadIdx.x & 31);
            const u64 key = i < n ? key_of(i) : 0ull;
            const bool in = key != 0ull && (key & mk) == pf;
            const unsigned d = in ? (unsigned)(key >> shift) & 255u : 256u;
            const unsigned same = __match_any_sync(0xffffffffu, d);
            if (in && (threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&st.hist[d], (unsigned)__popc(same));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // lane j owns digits 255-8j .. 248-8j (descending)
            const int lane = threadIdx.x;
            unsigned own = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) own += st.hist[255 - 8 * lane - b];
            unsigned incl = own;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned rem = (unsigned)st.remaining;
            const unsigned ballot = __ballot_sync(0xffffffffu, incl >= rem);
            if (ballot == 0u) {
                // fewer non-zero keys than K share the prefix: take them all (pass 0 only)
                if (lane == 0) {
                    st.done = 1;
                    st.prefix = 1ull;
                    st.mask = ~0ull;
                }
            } else if (lane == __ffs(ballot) - 1) {
                unsigned cum = incl - own;
                int d = 255 - 8 * lane;
                for (int b = 0; b < 8; ++b, --d) {
                    const unsigned h = st.hist[d];
                    if (cum + h >= rem) break;
                    cum += h;
                }
                const unsigned left = rem - cum;
                const u64 np = st.prefix | ((u64)d << shift);
                const u64 nm = st.mask | (0xFFull << shift);
                st.prefix = np;
                st.mask = nm;
                st.remaining = (int)left;
                if (st.hist[d] == left) st.done = 1;       // the whole bin is in
            }
        }
        __syncthreads();
        if (st.done) break;
    }
}

// cta_select_by over the array keys[0..n) (any address space)
static __device__ void cta_select(const u64* keys, int n, int K, SelState& st) {
    cta_select_by(n, K, st, [keys](int i) { return keys[i]; });
}

__device__ __forceinline__ bool selected(u64 key, const SelState& st) {
    return key != 0ull && (key & st.mask) >= st.prefix;
}

// The ft_peak records of image `img` from its cnt best keys sorted descending
// (sel[0..cnt)): (t, s) from the linear index, value = |P|, k = 2 (s - S/2) / S
// and b = t - H'/2 (eqs. 22-23); slots cnt .. K-1 zeroed; count[img] = cnt.
static __device__ void write_peaks(const u64* sel, int cnt, int K, int Hp, int S, ft_peak* out, int32_t* count,
                                   int img) {
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        ft_peak p;
        if (i < cnt) {
            const u64 key = sel[i];
            const unsigned lin = 0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull);
            p.t = (int)(lin / (unsigned)S);
            p.s = (int)(lin % (unsigned)S);
            p.value = __uint_as_float((unsigned)(key >> 32));
            p.k = 2.0f * (float)(p.s - S / 2) / (float)S;
            p.b = (float)(p.t - Hp / 2);
        } else {
            p.t = 0; p.s = 0; p.value = 0.f; p.k = 0.f; p.b = 0.f;
        }
        out[(size_t)img * K + i] = p;
    }
    if (threadIdx.x == 0) count[img] = cnt;
}

