// Device side of the library (sm_103a): the kernels of one homomorphic
// convolution layer and the plan / forward entry points of the C ABI.
//
// Pipeline of he_conv_forward (Sec. 2.3 hoisting, Sec. 3.1, Sec. 3.2.2):
//   1. k_ntt_inputs   NTT of c0, c1 and of the base-2^w digits of c1 of every
//                     input ciphertext (the "decompose once" half of hoisting)
//   2. k_keyswitch    per rotation: NTT-domain automorphism (an index
//                     permutation) of c0 and the digits, key inner product
//                     with lazy split sums and one reduction per sum
//   3. k_mac_tc       lazy CMult/HAdd over input channels, taps and diagonals
//                     on the tensor cores (exact fp16 chunks, fp32 sums), or
//      k_mac          on CUDA cores with 64-bit split accumulators (depthwise
//                     layers, |s| > 16, limbs of 2^50 or more); one reduction
//                     per sum; epilogue k*A0 + A1 * NTT(P_k) (the [k,-k] PMult).
//                     k_mac_eager is the conventional eager form, for ablations.
//   4. k_intt         inverse NTT to coefficient form
// Every stage kernel takes a table of layers, so one launch per stage runs a
// whole batch of layers (he_batch_*); a single layer is a table of one.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <memory>

#include "internal.h"

using namespace hy;

namespace {

// ------------------------------------------------------------------ constants
struct LimbC {
    u64 q, mu;       // Barrett constant for x < 2^(s+63)
    u32 sm1, delta;  // s - 1; delta = 2^50 - q if that is below 2^22 (else 0)
    u64 ninv, ninv_sh;
    u64 ksh;         // Shoup companion of the [k,-k] plaintext's k: floor(k 2^64 / q)
};
struct KP {
    u32 N, logN, L, l, w;
    u64 kmul;   // the k of the [k,-k] plaintext
    u64 kmul4;  // the k of the c_n = 4 patterns
    LimbC limb[HE_MAX_LIMBS];
    const u64* tw;   // [L][N][2]: psi^rev(k) and its Shoup companion, side by side (one 16-byte load)
    const u64* itw;  // [L][N][2]: psi^-rev(k) and its Shoup companion
};
struct RotDev {
    u32 galois, rot, key, galois_inv;  // galois_inv = galois^-1 mod 2N
};

// g^-1 mod 2N for odd g (Newton's iteration for inverses modulo a power of two: each step
// doubles the number of correct low bits; 5 steps from g (correct to 3 bits) reach 32 bits)
inline u32 galois_inverse(u32 g, u32 N) {
    u32 inv = g;
    for (int i = 0; i < 5; i++) inv *= 2u - g * inv;
    return inv & (2 * N - 1);
}

#define CUDA_OK(x)                                                                         \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ == cudaErrorMemoryAllocation) {                                              \
            cudaGetLastError();                                                            \
            fail(HE_ENOMEM, std::string(#x ": ") + cudaGetErrorString(e_));                \
        }                                                                                  \
        if (e_ != cudaSuccess) fail(HE_ECUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------ modular arithmetic
__device__ __forceinline__ u64 bred(u64 lo, u64 hi, const LimbC& m) {
    u64 q1 = (lo >> m.sm1) | (hi << (64 - m.sm1));
    u64 q3 = __umul64hi(q1, m.mu);
    u64 r = lo - q3 * m.q;
    r = r >= m.q ? r - m.q : r;
    r = r >= m.q ? r - m.q : r;
    return r;
}
__device__ __forceinline__ u64 bred128(u128 x, const LimbC& m) { return bred((u64)x, (u64)(x >> 64), m); }
__device__ __forceinline__ u64 mulmod(u64 a, u64 b, const LimbC& m) { return bred(a * b, __umul64hi(a, b), m); }
// a w mod q for w < q with its Shoup companion wsh = floor(w 2^64 / q), any a < 2^64 (Shoup's
// product: the quotient estimate mulhi(a, wsh) is exact or one short, so one subtraction remains)
__device__ __forceinline__ u64 mulmod_shoup(u64 a, u64 w, u64 wsh, u64 q) {
    const u64 r = a * w - __umul64hi(a, wsh) * q;
    return r >= q ? r - q : r;
}
// A = hi 2^30 + lo mod q, the tensor-core MAC's recombined chunk sums (|lo| < 2^46, |hi| < 2^36).
// For q = 2^50 - delta (delta < 2^22) the part of A above bit 50 folds down once: with hi = hh 2^20
// + hl, A = hh 2^50 + hl 2^30 + lo = hh delta + hl 2^30 + lo (mod q), a sum S with |S| < 2^51; then
// t = S + 4q lies in [0, 2^53) and t - floor(t / 2^50) q = floor(t / 2^50) delta + (t mod 2^50) is
// below q + 6 delta, one conditional subtraction from [0, q).  Other limbs: 128-bit Barrett.
__device__ __forceinline__ u64 tc_reduce(long long lo, long long hi, const LimbC& m) {
    if (m.delta) {
        const long long hh = hi >> 20;  // arithmetic: hi = hh 2^20 + hl, 0 <= hl < 2^20
        const long long hl = hi & 0xFFFFF;
        const long long S = hh * (long long)m.delta + (hl << 30) + lo;
        const u64 t = (u64)(S + 4 * (long long)m.q);
        const u64 r = t - (t >> 50) * m.q;
        return r >= m.q ? r - m.q : r;
    }
    const i128 a = (i128)lo + ((i128)hi << 30) + ((i128)m.q << 40);
    return bred128((u128)a, m);
}
__device__ __forceinline__ u64 addq(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}

// ------------------------------------------------------------------ NTT
// One CTA transforms one limb-polynomial of N words.  The slot index has
// log2 N bits; a "window" is 4 consecutive bit positions [lo, lo+4).  Each
// thread holds, in registers, the 16 elements whose indices differ only in
// the window, runs every butterfly stage of those bit positions, and
// exchanges through shared memory between windows: 3-4 round trips instead
// of log2 N.  Butterflies keep Harvey's lazy ranges ([0,4q) forward, [0,2q)
// inverse; q < 2^58 leaves the headroom) and Shoup products with
// precomputed w' = floor(w 2^64 / q).
//
// Forward (Cooley-Tukey, natural -> bit-reversed): the stage on bit p pairs
// indices that differ in bit p, group i = index >> (p+1), twiddle
// psi^rev(2^(logN-1-p) + i).  Inverse (Gentleman-Sande) runs the bits in the
// opposite order with psi^-rev(...) at the same position.
constexpr int NTT_E = 16;
constexpr int NTT_MAX_THREADS = 256;
// N = 16384 needs 132 KB of shared memory per transform, so one CTA fits an SM: it runs with
// 512 threads (two element sets each, 128 registers: the whole register file) to keep 16 warps
// resident, as two 256-thread CTAs do for N = 8192
constexpr int NTT_BIG_THREADS = 512;
constexpr u32 NTT_BIG_N = 16384;

__device__ __forceinline__ u32 spad(u32 i) { return i + (i >> 5); }  // one pad word per 32
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 wsh, u64 q) {
    return a * w - __umul64hi(a, wsh) * q;  // in [0, 2q)
}

__device__ __forceinline__ ulonglong2 twiddle(const u64* __restrict__ twp, u32 i) {
    return __ldg(reinterpret_cast<const ulonglong2*>(twp) + i);
}

template <int PE_TOP>
__device__ __forceinline__ void fwd_window(u64 (&x)[NTT_E], u32 base_hi, u32 lo, u32 logN, const u64* __restrict__ tw,
                                           u64 q, u64 q2) {
#pragma unroll
    for (int pe = PE_TOP; pe >= 0; pe--) {
        const u32 off = 1u << (logN - 1 - (lo + pe));
#pragma unroll
        for (int e = 0; e < NTT_E; e++) {
            if (e & (1 << pe)) continue;
            const int e2 = e | (1 << pe);
            const u32 i = off + ((u32)(e >> (pe + 1)) | (base_hi << (3 - pe)));
            const ulonglong2 w = twiddle(tw, i);
            const u64 W = w.x, Ws = w.y;
            u64 X = x[e];
            X = X >= q2 ? X - q2 : X;
            const u64 T = shoup_lazy(x[e2], W, Ws, q);
            x[e] = X + T;
            x[e2] = X - T + q2;
        }
    }
}

template <int PE_BOT>
__device__ __forceinline__ void inv_window(u64 (&x)[NTT_E], u32 base_hi, u32 lo, u32 logN, const u64* __restrict__ itw,
                                           u64 q, u64 q2) {
#pragma unroll
    for (int pe = PE_BOT; pe <= 3; pe++) {
        const u32 off = 1u << (logN - 1 - (lo + pe));
#pragma unroll
        for (int e = 0; e < NTT_E; e++) {
            if (e & (1 << pe)) continue;
            const int e2 = e | (1 << pe);
            const u32 i = off + ((u32)(e >> (pe + 1)) | (base_hi << (3 - pe)));
            const ulonglong2 w = twiddle(itw, i);
            const u64 W = w.x, Ws = w.y;
            const u64 X = x[e], Y = x[e2];
            const u64 S = X + Y;
            x[e] = S >= q2 ? S - q2 : S;
            x[e2] = shoup_lazy(X - Y + q2, W, Ws, q);
        }
    }
}

// index of element e of set `set` in window [lo, lo+4)
__device__ __forceinline__ u32 win_base(u32 set, u32 lo) { return ((set >> lo) << (lo + 4)) | (set & ((1u << lo) - 1)); }

// Forward NTT of one polynomial: load(i) gives coefficient i in [0, 4q); store(i, v) receives slot i in [0, q).
template <class Load, class Store>
__device__ void ntt_forward_block(u64* sm, u32 N, u32 logN, const u64* tw, u64 q, Load load,
                                  Store store) {
    const u64 q2 = 2 * q;
    const u32 sets = N / NTT_E;
    u64 x[NTT_E];
    // first window: bits [logN-4, logN), loaded straight from global (coalesced: stride N/16)
    u32 lo = logN - 4;
    for (u32 set = threadIdx.x; set < sets; set += blockDim.x) {
#pragma unroll
        for (int e = 0; e < NTT_E; e++) x[e] = load(set | ((u32)e << lo));
        fwd_window<3>(x, 0, lo, logN, tw, q, q2);
        if (lo == 0) {
#pragma unroll
            for (int e = 0; e < NTT_E; e++) {
                u64 v = x[e];
                v = v >= q2 ? v - q2 : v;
                store(set | ((u32)e << lo), v >= q ? v - q : v);
            }
        } else {
#pragma unroll
            for (int e = 0; e < NTT_E; e++) sm[spad(set | ((u32)e << lo))] = x[e];
        }
    }
    while (lo > 0) {
        const u32 nlo = lo > 4 ? lo - 4 : 0;
        const int pe_top = (int)(lo - 1 - nlo);
        __syncthreads();
        for (u32 set = threadIdx.x; set < sets; set += blockDim.x) {
            const u32 base = win_base(set, nlo);
#pragma unroll
            for (int e = 0; e < NTT_E; e++) x[e] = sm[spad(base | ((u32)e << nlo))];
            const u32 bh = base >> (nlo + 4);
            switch (pe_top) {
                case 3: fwd_window<3>(x, bh, nlo, logN, tw, q, q2); break;
                case 2: fwd_window<2>(x, bh, nlo, logN, tw, q, q2); break;
                case 1: fwd_window<1>(x, bh, nlo, logN, tw, q, q2); break;
                default: fwd_window<0>(x, bh, nlo, logN, tw, q, q2); break;
            }
            if (nlo == 0) {
#pragma unroll
                for (int e = 0; e < NTT_E; e++) {
                    u64 v = x[e];
                    v = v >= q2 ? v - q2 : v;
                    store(base | (u32)e, v >= q ? v - q : v);
                }
            } else {
                // a set writes back exactly the positions it read, and sets are disjoint
#pragma unroll
                for (int e = 0; e < NTT_E; e++) sm[spad(base | ((u32)e << nlo))] = x[e];
            }
        }
        lo = nlo;
    }
}

// Inverse NTT (with the 1/N factor): load(i) gives slot i in [0, 2q); store(i, v) receives coefficient i in [0, q).
template <class Load, class Store>
__device__ void ntt_inverse_block(u64* sm, u32 N, u32 logN, const u64* itw, u64 q, u64 ninv,
                                  u64 ninv_sh, Load load, Store store) {
    const u64 q2 = 2 * q;
    const u32 sets = N / NTT_E;
    u64 x[NTT_E];
    u32 lo = 0;  // windows [0,4), [4,8), ...; the last one is [logN-4, logN) starting at the first unfinished bit
    bool first = true;
    while (true) {
        const u32 wlo = (lo + 4 <= logN) ? lo : logN - 4;
        const int pe_bot = (int)(lo - wlo);
        const bool last = wlo + 4 >= logN;
        if (!first) __syncthreads();
        for (u32 set = threadIdx.x; set < sets; set += blockDim.x) {
            const u32 base = win_base(set, wlo);
            if (first) {
#pragma unroll
                for (int e = 0; e < NTT_E; e++) x[e] = load(base | ((u32)e << wlo));
            } else {
#pragma unroll
                for (int e = 0; e < NTT_E; e++) x[e] = sm[spad(base | ((u32)e << wlo))];
            }
            const u32 bh = base >> (wlo + 4);
            switch (pe_bot) {
                case 0: inv_window<0>(x, bh, wlo, logN, itw, q, q2); break;
                case 1: inv_window<1>(x, bh, wlo, logN, itw, q, q2); break;
                case 2: inv_window<2>(x, bh, wlo, logN, itw, q, q2); break;
                default: inv_window<3>(x, bh, wlo, logN, itw, q, q2); break;
            }
            if (last) {
#pragma unroll
                for (int e = 0; e < NTT_E; e++) {
                    u64 v = shoup_lazy(x[e], ninv, ninv_sh, q);
                    store(base | ((u32)e << wlo), v >= q ? v - q : v);
                }
            } else {
#pragma unroll
                for (int e = 0; e < NTT_E; e++) sm[spad(base | ((u32)e << wlo))] = x[e];
            }
        }
        if (last) break;
        first = false;
        lo = wlo + 4;
    }
}

__host__ __device__ constexpr size_t ntt_smem_bytes(u32 N) { return ((size_t)N + N / 32) * 8; }

// ------------------------------------------------------------------ batched launches
// Every stage kernel runs over a table of layers passed by value: block b of a
// launch belongs to the layer l with start[stage][l] <= b < start[stage][l+1]
// (binary search; empty layers are skipped) and works on local block
// b - start[stage][l].  A single layer is a table of one.
struct LayerDev {
    CUtensorMap rmap;          // R as a 3-D tensor (slot, polynomial*L + limb, row = ct*n_rot + rot), tensor-core MAC;
                               // CTA-pair MAC: the operand images (tcp_encode_maps)
    CUtensorMap smap;          // CTA-pair MAC: the scalar tiles
    const u64* in;             // input ciphertexts [n_ct_in][2][L][N]
    u64* R;                    // rotated copies [n_ct_in][n_rot][2][L][N], NTT form
    u64* D;                    // digit NTTs [n_ct_in][L l][L][N], each word split at bit 25 (low bits | rest << 32)
    u64* O;                    // NTT-form outputs [n_ct_out][2][L][N]
    u64* out;                  // output ciphertexts [n_ct_out][2][L][N]
    const u64* isrc;           // inverse-NTT source (O, or a rotated copy for he_rotate)
    unsigned long long isrc_stride;  // words between the inverse-NTT source ciphertexts
    const u64* ksk;            // Galois keys [n_gal][L l][2][L][N], NTT form
    const RotDev* rots;        // rotations that need a key switch
    const int16_t* scal;       // CUDA-core MAC scalars [out_groups][c_n][K]
    const u64* pk;             // NTT(P_k) [L][N]
    const u64* pksh;           // Shoup companions floor(NTT(P_k) 2^64 / q) [L][N]
    const __half* sc16;        // tensor-core MAC scalars, one shared-memory tile image per (row tile, K tile)
    const int* bias;           // tensor-core MAC row offsets 512 sum(s)
    int* err;                  // bounded-wait status
    u32 n_ct_in, n_ct_out, n_rot, rot_id, n_ks, K, Kpad, in_groups, out_groups, row_units, tc_rows, tc_rows_per_cta;
    u32 tmem_cols;             // TMEM columns of a tensor-core MAC CTA (power of two >= 5 rows)
    u32 r_slots, r_id;         // rotated copies stored per input ciphertext in R, and the identity's slot
    // operand-image form (tensor-core MAC fed with ready fp16 chunk images, see k_keyswitch_img)
    __half* A16;               // images [row_units][2][L][N/128][ktiles][5 chunks][128 slots x 32 terms]
    const RotDev* rots_all;    // every rotation of the layer, identity included (key = ~0u)
    u32 img, in_pad, n_rot_all, id_rot;  // in_pad = in_groups rounded up to 8; id_rot = the identity's index
    u32 ks_rg;                 // rotation groups of the image key switch (ksi_groups)
    u32 fused;                 // key switch inside the MAC (k_ksmac): no image buffer, no key-switch launch
};

enum { ST_NTT = 0, ST_KS = 1, ST_MAC = 2, ST_INTT = 3 };

template <int MAXB>
struct Batch {
    u32 n;
    u32 start[4][MAXB + 1];
    LayerDev L[MAXB];
};

template <int MAXB>
__device__ __forceinline__ u32 find_layer(const Batch<MAXB>& B, int stage, u32 blk) {
    if (MAXB == 1) return 0;
    u32 lo = 0, hi = B.n;  // last l with start[l] <= blk
    while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (B.start[stage][mid] <= blk) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Step 1: forward NTT of the inputs.  Local block = (c, job): job < 2L ->
// polynomial job/L, limb job%L into R[c][rot_id]; otherwise digit
// dd = (job-2L)/L of c1 lifted into limb (job-2L)%L, into D[c][dd].  Digits
// are below 2^w <= 2^s < 2q, inside the forward transform's input range.
template <int MAXB, int NTHR, int MINB>
__global__ void __launch_bounds__(NTHR, MINB) k_ntt_inputs(const __grid_constant__ Batch<MAXB> B, KP kp) {
    extern __shared__ u64 sm[];
    const u32 li = find_layer(B, ST_NTT, blockIdx.x);
    const LayerDev& Ly = B.L[li];
    const u32 N = kp.N, L = kp.L, l = kp.l;
    // with one digit per limb (l = 1) the digit of c1 in its own limb is c1 itself, so the
    // NTT of c1 is not a job of its own: the digit job (dd = k, limb k) also writes it to R
    const u32 c1_jobs = l == 1 ? 0 : L;
    const u32 jobs = L + c1_jobs + L * l * L;
    const u32 local = blockIdx.x - B.start[ST_NTT][li];
    const u32 c = local / jobs, y = local % jobs;
    const size_t ctw = 2ull * L * N;
    u64* const Rid = Ly.R + ((size_t)c * Ly.r_slots + Ly.r_id) * ctw;
    const u64* src;
    u64* dst;
    u64* dst2 = nullptr;
    u32 limb, shift = 0;
    u64 mask = ~0ull;
    bool split = false;  // digit transforms are stored split at bit 25 (see k_keyswitch)
    if (y < L + c1_jobs) {
        limb = y % L;
        src = Ly.in + c * ctw + (size_t)y * N;
        dst = Rid + (size_t)y * N;
    } else {
        split = true;
        const u32 z = y - L - c1_jobs, dd = z / L;
        limb = z % L;
        src = Ly.in + c * ctw + (size_t)(L + dd / l) * N;
        dst = Ly.D + (((size_t)c * L * l + dd) * L + limb) * N;
        shift = kp.w * (dd % l);
        mask = (kp.w >= 64) ? ~0ull : ((1ull << kp.w) - 1);
        if (l == 1 && dd == limb) dst2 = Rid + (size_t)(L + limb) * N;
    }
    const LimbC m = kp.limb[limb];
    ntt_forward_block(
        sm, N, kp.logN, kp.tw + 2 * (size_t)limb * N, m.q,
        [&](u32 i) { return shift >= 64 ? 0ull : (__ldg(src + i) >> shift) & mask; },
        [&](u32 i, u64 v) {
            dst[i] = split ? (v & 0x1FFFFFFull) | ((v >> 25) << 32) : v;
            if (dst2) dst2[i] = v;
        });
}

// Plain batched NTT: polynomial blockIdx.x of [n][N], limb = index % L.
__global__ void __launch_bounds__(NTT_MAX_THREADS) k_ntt_plain(u64* __restrict__ a, KP kp, int inverse) {
    extern __shared__ u64 sm[];
    const u32 N = kp.N, limb = blockIdx.x % kp.L;
    u64* poly = a + (size_t)blockIdx.x * N;
    const LimbC m = kp.limb[limb];
    if (!inverse)
        ntt_forward_block(sm, N, kp.logN, kp.tw + 2 * (size_t)limb * N, m.q,
                          [&](u32 i) { return poly[i]; }, [&](u32 i, u64 v) { poly[i] = v; });
    else
        ntt_inverse_block(sm, N, kp.logN, kp.itw + 2 * (size_t)limb * N, m.q, m.ninv,
                          m.ninv_sh, [&](u32 i) { return poly[i]; }, [&](u32 i, u64 v) { poly[i] = v; });
}

// Step 4: inverse NTT of the outputs.  Local block = (ciphertext, polynomial*L + limb).
template <int MAXB, int NTHR, int MINB>
__global__ void __launch_bounds__(NTHR, MINB) k_intt(const __grid_constant__ Batch<MAXB> B, KP kp) {
    extern __shared__ u64 sm[];
    const u32 li = find_layer(B, ST_INTT, blockIdx.x);
    const LayerDev& Ly = B.L[li];
    const u32 N = kp.N, L = kp.L;
    const u32 local = blockIdx.x - B.start[ST_INTT][li];
    const u32 c = local / (2 * L), y = local % (2 * L), limb = y % L;
    const u64* s = Ly.isrc + c * Ly.isrc_stride + (size_t)y * N;
    u64* d = Ly.out + c * (2ull * L * N) + (size_t)y * N;
    const LimbC m = kp.limb[limb];
    ntt_inverse_block(sm, N, kp.logN, kp.itw + 2 * (size_t)limb * N, m.q, m.ninv,
                      m.ninv_sh, [&](u32 i) { return __ldg(s + i); }, [&](u32 i, u64 v) { d[i] = v; });
}

// Barrett reduction of x = hi 2^50 + mid 2^25 + lo for a 50-bit limb (s - 1 = 49), without 128-bit
// arithmetic: lo < 2^58, mid < 2^56, hi < 2^55 (at most 16 digit terms), so x < 2^106 < 2^(s+63) and
//   floor(x / 2^49) = 2 hi + floor(mid / 2^24) + floor(((mid mod 2^24) 2^25 + lo) / 2^49)
// with the last numerator below 2^59.  The quotient estimate mulhi(q1, mu) is the same as bred's.
__device__ __forceinline__ u64 bred_split50(u64 lo, u64 mid, u64 hi, const LimbC& m) {
    const u64 t = ((mid & 0xFFFFFFull) << 25) + lo;
    const u64 q1 = (hi << 1) + (mid >> 24) + (t >> 49);
    const u64 xlo = lo + (mid << 25) + (hi << 50);  // x mod 2^64
    const u64 q3 = __umul64hi(q1, m.mu);
    u64 r = xlo - q3 * m.q;
    r = r >= m.q ? r - m.q : r;
    r = r >= m.q ? r - m.q : r;
    return r;
}

// The same sum x = hi 2^50 + mid 2^25 + lo modulo q = 2^50 - delta (0 < delta < 2^22), without a
// 64x64-bit product: 2^50 = delta (mod q), so the part of x above bit 50 folds down as a multiple of
// delta, twice, with 32x32-bit products.  lo < 2^55, mid < 2^56, hi < 2^55 (at most 16 digit terms).
//   x = A 2^50 + B                 A = hi + mid / 2^25 + carry < 2^55,  B < 2^50
//     = A delta + B = C 2^50 + D   (A delta split at bit 32, the high product folded again)
//     = C delta + D = z  < 1.5 2^50 < 2q
__device__ __forceinline__ u64 fold_reduce50(u64 lo, u64 mid, u64 hi, const LimbC& m) {
    const u64 M50 = (1ull << 50) - 1;
    u64 A = hi + (mid >> 25);
    u64 B = ((mid & 0x1FFFFFFull) << 25) + lo;
    A += B >> 50;
    B &= M50;
    const u32 d = m.delta;
    const u64 P0 = (u64)(u32)A * d;          // < 2^54
    const u64 P1 = (u64)(u32)(A >> 32) * d;  // < 2^45
    u64 C = P1 >> 18;
    u64 D = ((P1 & 0x3FFFFull) << 32) + P0 + B;
    C += D >> 50;
    D &= M50;
    const u64 z = (u64)(u32)C * d + D;
    return z >= m.q ? z - m.q : z;
}

// acc += a * b with one unsigned 32x32 -> 64-bit multiply-add
__device__ __forceinline__ void mad_wide_u(u64& acc, u32 a, u32 b) {
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// Step 2: hoisted key switch.  Local block = (rotation, limb, slot tile).
// The NTT slot x holds the evaluation at psi^e with e = 2 rev(x) + 1, so
// sigma_g(a)[x] = a[src(x)] with src(x) = rev((g e(x) mod 2N - 1)/2).  A thread owns a
// SOURCE slot y of the tile and writes the destination x = src^-1(y) = rev((g^-1 e(y) mod
// 2N - 1)/2): its loads of the digit and c0 transforms are coalesced, only its two stores
// are permuted (within one aligned tile, since the map keeps the tile).  The key values of
// (x, limb) stay in registers across all input ciphertexts of the layer.
constexpr int KS_THREADS = 256;
template <int LL, int MAXB>
__global__ void __launch_bounds__(KS_THREADS) k_keyswitch(const __grid_constant__ Batch<MAXB> B, KP kp) {
    const u32 li = find_layer(B, ST_KS, blockIdx.x);
    const LayerDev& Ly = B.L[li];
    const u32 N = kp.N, L = kp.L, logN = kp.logN;
    const u32 xt_n = N / KS_THREADS;
    const u32 local = blockIdx.x - B.start[ST_KS][li];
    const u32 xt = local % xt_n, k = (local / xt_n) % L, r = local / (xt_n * L);
    const u32 src = xt * KS_THREADS + threadIdx.x;
    const RotDev rd = Ly.rots[r];
    const LimbC m = kp.limb[k];
    const u32 e = 2 * (__brev(src) >> (32 - logN)) + 1;
    const u32 e2 = (u32)(((u64)e * rd.galois_inv) & (2ull * N - 1));
    const u32 x = __brev((e2 - 1) >> 1) >> (32 - logN);
    // keys split at bit 25, held in registers for all input ciphertexts: a product of two
    // residues below 2^s is (a1 2^25 + a0)(b1 2^25 + b0), four 32x32 -> 64-bit multiply-adds
    // into three 64-bit partial sums.  With s <= 54 and at most 16 digit terms the high halves
    // fit 32 bits and every partial sum stays below 2^64; the recombined sum is below 2^113.
    u32 k0l[LL], k0h[LL], k1l[LL], k1h[LL];
    const u64* kb = Ly.ksk + (size_t)rd.key * LL * 2 * L * N;
#pragma unroll
    for (int dd = 0; dd < LL; dd++) {
        const u64 a = kb[(((size_t)dd * 2 + 0) * L + k) * N + x], b = kb[(((size_t)dd * 2 + 1) * L + k) * N + x];
        k0l[dd] = (u32)(a & 0x1FFFFFFu), k0h[dd] = (u32)(a >> 25);
        k1l[dd] = (u32)(b & 0x1FFFFFFu), k1h[dd] = (u32)(b >> 25);
    }
    const size_t ctw = 2ull * L * N;
    const u32 r_slots = Ly.r_slots, r_id = Ly.r_id;
    if (m.sm1 == 49) {
        // 50-bit limbs: halves below 2^25, so the Karatsuba middle term (a0 + a1)(b0 + b1) - a0 b0 - a1 b1
        // needs one multiply-add per product instead of two; its factors stay below 2^26 and the sums of
        // at most 16 digit terms below 2^57.  The two subtractions are taken once per sum.
        u32 k0s[LL], k1s[LL];
#pragma unroll
        for (int dd = 0; dd < LL; dd++) k0s[dd] = k0l[dd] + k0h[dd], k1s[dd] = k1l[dd] + k1h[dd];
#pragma unroll 4
        for (u32 c = 0; c < Ly.n_ct_in; c++) {
            const u64* Dc = Ly.D + (size_t)c * LL * L * N + (size_t)k * N + src;
            u64 lo0 = 0, mid0 = 0, hi0 = 0, lo1 = 0, mid1 = 0, hi1 = 0;
#pragma unroll
            for (int dd = 0; dd < LL; dd++) {
                const u64 dv = __ldg(Dc + (size_t)dd * L * N);
                const u32 dl = (u32)dv, dh = (u32)(dv >> 32), ds = dl + dh;  // stored split at bit 25
                mad_wide_u(lo0, dl, k0l[dd]);
                mad_wide_u(hi0, dh, k0h[dd]);
                mad_wide_u(mid0, ds, k0s[dd]);
                mad_wide_u(lo1, dl, k1l[dd]);
                mad_wide_u(hi1, dh, k1h[dd]);
                mad_wide_u(mid1, ds, k1s[dd]);
            }
            mid0 -= lo0 + hi0;
            mid1 -= lo1 + hi1;
            u64* Rc = Ly.R + (size_t)c * r_slots * ctw;
            lo0 += __ldg(Rc + (size_t)r_id * ctw + (size_t)k * N + src);  // + sigma(c0); lo stays below 2^57
            u64 r0, r1;
            if (m.delta) {
                r0 = fold_reduce50(lo0, mid0, hi0, m);
                r1 = fold_reduce50(lo1, mid1, hi1, m);
            } else {
                r0 = bred_split50(lo0, mid0, hi0, m);
                r1 = bred_split50(lo1, mid1, hi1, m);
            }
            // R streams out once and is read once by the MAC: evict-first keeps D and the keys in L2
            __stcs(reinterpret_cast<unsigned long long*>(Rc + (size_t)rd.rot * ctw + (size_t)k * N + x), r0);
            __stcs(reinterpret_cast<unsigned long long*>(Rc + (size_t)rd.rot * ctw + (size_t)(L + k) * N + x), r1);
        }
        return;
    }
#pragma unroll 2
    for (u32 c = 0; c < Ly.n_ct_in; c++) {
        const u64* Dc = Ly.D + (size_t)c * LL * L * N + (size_t)k * N + src;
        u64 lo0 = 0, mid0 = 0, hi0 = 0, lo1 = 0, mid1 = 0, hi1 = 0;
#pragma unroll
        for (int dd = 0; dd < LL; dd++) {
            const u64 dv = __ldg(Dc + (size_t)dd * L * N);
            const u32 dl = (u32)dv, dh = (u32)(dv >> 32);  // stored split at bit 25
            mad_wide_u(lo0, dl, k0l[dd]);
            mad_wide_u(mid0, dl, k0h[dd]);
            mad_wide_u(mid0, dh, k0l[dd]);
            mad_wide_u(hi0, dh, k0h[dd]);
            mad_wide_u(lo1, dl, k1l[dd]);
            mad_wide_u(mid1, dl, k1h[dd]);
            mad_wide_u(mid1, dh, k1l[dd]);
            mad_wide_u(hi1, dh, k1h[dd]);
        }
        u64* Rc = Ly.R + (size_t)c * r_slots * ctw;
        lo0 += __ldg(Rc + (size_t)r_id * ctw + (size_t)k * N + src);
        const u64 r0 = bred128(((u128)hi0 << 50) + ((u128)mid0 << 25) + lo0, m);
        const u64 r1 = bred128(((u128)hi1 << 50) + ((u128)mid1 << 25) + lo1, m);
        __stcs(reinterpret_cast<unsigned long long*>(Rc + (size_t)rd.rot * ctw + (size_t)k * N + x), r0);
        __stcs(reinterpret_cast<unsigned long long*>(Rc + (size_t)rd.rot * ctw + (size_t)(L + k) * N + x), r1);
    }
}

// Step 3: lazy channel multiply-accumulate (CMult^- and HAdd^128 of Sec. 3.2.2).
// Each residue v < 2^50 is split v = vh 2^25 + vl; s*vl and s*vh accumulate
// exactly in int64 (|s| <= 2^15, at most 2^14 terms), and A = hi 2^25 + lo is
// reduced once.  NR rows per output group: NR = 2, the Walsh-Hadamard pair with the
// epilogue out = k*[A0] + [A1] * NTT(P_k); NR = 4, the 4 x 4 basis with
// out = k4*[A0] + sum_b [A_b] * NTT(k4 pattern_b); NR = 1, out = [A0].
constexpr int MAC_THREADS = 256;
constexpr int MAC_KC = 128;

__device__ __forceinline__ u64 reduce_split(i64 lo, i64 hi, const LimbC& m) {
    i128 a = ((i128)hi << 25) + (i128)lo + ((i128)m.q << 32);
    return bred128((u128)a, m);
}

// acc += a * b with one 32x32 -> 64-bit signed multiply-add
__device__ __forceinline__ void mad_wide(i64& acc, int a, int b) {
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// Local block = ((row unit, polynomial, limb), slot tile, group tile); the
// group tile varies fastest so that blocks reading the same residues run together.
template <int GT, int NR, bool DW, int MAXB>
__global__ void __launch_bounds__(MAC_THREADS) k_mac(const __grid_constant__ Batch<MAXB> B, KP kp) {
    static_assert(NR == 1 || NR == 2 || NR == 4, "rows per output group: 1, 2 or 4");
    constexpr int NS = GT * NR;            // scalars used per term
    constexpr int NSP = (NS + 3) & ~3;     // padded to whole int4 loads
    __shared__ __align__(16) int ss[MAC_KC][NSP];
    const u32 li = find_layer(B, ST_MAC, blockIdx.x);
    const LayerDev& Ly = B.L[li];
    const u32 N = kp.N, L = kp.L;
    const u32 gtiles = (Ly.out_groups + GT - 1) / GT, xt_n = N / MAC_THREADS;
    const u32 local = blockIdx.x - B.start[ST_MAC][li];
    const u32 gt = local % gtiles, xt = (local / gtiles) % xt_n, z = local / (gtiles * xt_n);
    const u32 x = xt * MAC_THREADS + threadIdx.x;
    const u32 g0 = gt * GT;
    const u32 k = z % L, p = (z / L) & 1, ru = z / (2 * L);
    const LimbC m = kp.limb[k];
    const size_t ctw = 2ull * L * N;
    const u32 K = Ly.K, n_rot = Ly.n_rot, in_groups = Ly.in_groups, out_groups = Ly.out_groups;
    i64 lo[NS], hi[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) lo[i] = hi[i] = 0;

    for (u32 kc0 = 0; kc0 < K; kc0 += MAC_KC) {
        const u32 kcn = min((u32)MAC_KC, K - kc0);
        for (u32 idx = threadIdx.x; idx < (u32)(MAC_KC * NSP); idx += MAC_THREADS) {
            const u32 kk = idx / NSP, c = idx % NSP, g = c / NR, r = c % NR;
            int v = 0;
            if (kk < kcn && c < (u32)NS && g0 + g < out_groups) v = Ly.scal[((size_t)(g0 + g) * NR + r) * K + kc0 + kk];
            ss[kk][c] = v;
        }
        __syncthreads();
        const u64* base = Ly.R + ((size_t)p * L + k) * N + x;
#pragma unroll 2
        for (u32 kk = 0; kk < kcn; kk++) {
            const u32 kg = kc0 + kk;
            // depthwise: the term's input ciphertext is phase kg / n_rot of output group g0
            // (one phase unless polyphase packing gives four)
            const u32 ct = DW ? ru * in_groups + (kg / n_rot) * out_groups + g0 : ru * in_groups + kg / n_rot;
            const u32 rot = kg % n_rot;
            const u64 v = __ldg(base + ((size_t)ct * n_rot + rot) * ctw);
            const int vl = (int)(v & 0x1FFFFFFull), vh = (int)(v >> 25);
            int sv[NSP];
#pragma unroll
            for (int i = 0; i < NSP; i += 4) {
                const int4 q4 = *reinterpret_cast<const int4*>(&ss[kk][i]);
                sv[i] = q4.x, sv[i + 1] = q4.y, sv[i + 2] = q4.z, sv[i + 3] = q4.w;
            }
#pragma unroll
            for (int i = 0; i < NS; i++) {
                mad_wide(lo[i], sv[i], vl);
                mad_wide(hi[i], sv[i], vh);
            }
        }
        __syncthreads();
    }
    // NTT of the pattern plaintexts at this slot: pk [NR - 1][L][N]
    u64 pkv[NR > 1 ? NR - 1 : 1];
#pragma unroll
    for (int b = 0; b < NR - 1; b++) pkv[b] = Ly.pk[((size_t)b * L + k) * N + x];
#pragma unroll
    for (int g = 0; g < GT; g++) {
        if (g0 + g >= out_groups) break;
        u64 out = reduce_split(lo[g * NR], hi[g * NR], m);
        if (NR > 1) {
            out = mulmod(NR == 2 ? kp.kmul : kp.kmul4, out, m);
#pragma unroll
            for (int b = 1; b < NR; b++)
                out = addq(out, mulmod(reduce_split(lo[g * NR + b], hi[g * NR + b], m), pkv[b - 1], m), m.q);
        }
        Ly.O[((size_t)(ru * out_groups + g0 + g) * 2 + p) * L * N + (size_t)k * N + x] = out;
    }
}

// Eager form, for the ablation of Sec. 3.2.2 only: the same tiling and scalar staging as
// k_mac (GT = 4 groups), but every CMult is reduced (Barrett on the full product) and
// every HAdd is a modular add, as a conventional implementation does.  Same outputs.
template <bool PACKED, int MAXB>
__global__ void __launch_bounds__(MAC_THREADS) k_mac_eager(const __grid_constant__ Batch<MAXB> B, KP kp) {
    constexpr int GT = 4, NR = PACKED ? 2 : 1, NS = GT * NR, NSP = (NS + 3) & ~3;
    __shared__ __align__(16) int ss[MAC_KC][NSP];
    const u32 li = find_layer(B, ST_MAC, blockIdx.x);
    const LayerDev& Ly = B.L[li];
    const u32 N = kp.N, L = kp.L;
    const u32 gtiles = (Ly.out_groups + GT - 1) / GT, xt_n = N / MAC_THREADS;
    const u32 local = blockIdx.x - B.start[ST_MAC][li];
    const u32 gt = local % gtiles, xt = (local / gtiles) % xt_n, z = local / (gtiles * xt_n);
    const u32 x = xt * MAC_THREADS + threadIdx.x, g0 = gt * GT;
    const u32 k = z % L, p = (z / L) & 1, ru = z / (2 * L);
    const LimbC m = kp.limb[k];
    const size_t ctw = 2ull * L * N;
    const u32 K = Ly.K, n_rot = Ly.n_rot, in_groups = Ly.in_groups, out_groups = Ly.out_groups;
    u64 acc[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) acc[i] = 0;
    for (u32 kc0 = 0; kc0 < K; kc0 += MAC_KC) {
        const u32 kcn = min((u32)MAC_KC, K - kc0);
        for (u32 idx = threadIdx.x; idx < (u32)(MAC_KC * NSP); idx += MAC_THREADS) {
            const u32 kk = idx / NSP, c = idx % NSP, g = c / NR, r = c % NR;
            int v = 0;
            if (kk < kcn && c < (u32)NS && g0 + g < out_groups) v = Ly.scal[((size_t)(g0 + g) * NR + r) * K + kc0 + kk];
            ss[kk][c] = v;
        }
        __syncthreads();
        const u64* base = Ly.R + ((size_t)p * L + k) * N + x;
#pragma unroll 2
        for (u32 kk = 0; kk < kcn; kk++) {
            const u32 kg = kc0 + kk;
            const u32 ct = ru * in_groups + kg / n_rot, rot = kg % n_rot;
            const u64 v = __ldg(base + ((size_t)ct * n_rot + rot) * ctw);
            int sv[NSP];
#pragma unroll
            for (int i = 0; i < NSP; i += 4) {
                const int4 q4 = *reinterpret_cast<const int4*>(&ss[kk][i]);
                sv[i] = q4.x, sv[i + 1] = q4.y, sv[i + 2] = q4.z, sv[i + 3] = q4.w;
            }
#pragma unroll
            for (int i = 0; i < NS; i++) {
                const u64 prod = mulmod((u64)(sv[i] < 0 ? -sv[i] : sv[i]), v, m);  // CMult, reduced
                acc[i] = sv[i] < 0 ? (acc[i] >= prod ? acc[i] - prod : acc[i] + m.q - prod)
                                   : addq(acc[i], prod, m.q);                     // HAdd, reduced
            }
        }
        __syncthreads();
    }
    const u64 pkv = PACKED ? Ly.pk[(size_t)k * N + x] : 0;
#pragma unroll
    for (int g = 0; g < GT; g++) {
        if (g0 + g >= out_groups) break;
        u64 out = acc[g * NR];
        if (PACKED) out = addq(mulmod(kp.kmul, out, m), mulmod(acc[g * NR + 1], pkv, m), m.q);
        Ly.O[((size_t)(ru * out_groups + g0 + g) * 2 + p) * L * N + (size_t)k * N + x] = out;
    }
}

// ------------------------------------------------------------------ tensor-core MAC (tcgen05)
// The same contraction on the 5th-generation tensor cores.  Rows of rotated
// residues stream into shared memory by bulk asynchronous copies (TC_RAW tiles
// in flight), are split into fp16 chunks by all threads, and feed the MMA,
// which one thread issues.  Per CTA tile:
//   D_c[n][m] = sum_kk (x_c(n, kk) - 512) * s(m, kk),  c = 0..4,
// n = 128 NTT slots (MMA M), m = output rows (g, r) (MMA N, <= 96),
// kk = (input ciphertext, rotation) terms (MMA K), x_c = 10-bit chunk c of the
// residue.  Operands are fp16 (exact integers), accumulators fp32 in TMEM:
// |s| <= 16 and |x_c - 512| <= 512 keep every partial sum below 2^24 for
// 2048 terms, so the fp32 sums are exact integers.  Longer contractions run
// as segments of at most 2048 terms, each accumulated afresh in TMEM.  The
// epilogue of a segment forms
//   A = sum_c 2^(10c) (D_c + 512 S),  S = sum of the segment's s,
// (each chunk's sum plus 512 S stays below 2^25), reduces it once mod q_k and
// applies the [k,-k] PMult as in k_mac; since that map is linear, segment
// results add mod q_k into the output, which the same thread wrote before.
// Shared-memory operands use the no-swizzle K-major canonical layout: 8x16-byte
// core matrices, LBO = 128 B between core matrices along K, SBO = 512 B
// between core matrices along M/N (a 32-term K tile is 4 core matrices wide).
constexpr int TC_THREADS = 512;
constexpr int TC_MTILE = 128;     // NTT slots per CTA (MMA M)
constexpr int TC_KTILE = 32;      // terms per pipeline stage
constexpr int TC_CHUNKS = 5;      // 10-bit chunks of a residue < 2^50
constexpr int TC_NMAX = 96;       // output rows per CTA (MMA N <= 96 so 5 N <= 512 TMEM columns)
constexpr int TC_KMAX = 2048;     // exactness bound on the terms of one fp32 accumulation for |s| <= 16
constexpr u32 TC_SEG_TILES = TC_KMAX / TC_KTILE;  // K tiles per accumulation segment
constexpr int TC_SMAX = 16;
constexpr u32 TC_A_CHUNK_BYTES = TC_MTILE * TC_KTILE * 2;          // 8 KB
constexpr u32 TC_A_BYTES = TC_CHUNKS * TC_A_CHUNK_BYTES;           // 40 KB
constexpr u32 TC_B_BYTES = TC_NMAX * TC_KTILE * 2;                 // 6 KB
constexpr u32 TC_SBO = (TC_KTILE / 8) * 128;                       // bytes between 8-row core-matrix blocks
constexpr u32 TC_STAGE_BYTES = TC_A_BYTES;                         // converted residues, 2 stages
constexpr int TC_RAW = 3;                                          // raw residue tiles (TC_RAW - 1 in flight)
constexpr u32 TC_RAW_BYTES = TC_KTILE * TC_MTILE * 8;              // 32 KB: 32 rows of 128 residues
constexpr u32 TC_RAW_OFF = 2 * TC_STAGE_BYTES;
constexpr u32 TC_BS_OFF = TC_RAW_OFF + TC_RAW * TC_RAW_BYTES;
constexpr u32 TC_BAR_OFF = TC_BS_OFF + TC_RAW * TC_B_BYTES;         // scalar tile of slot s at TC_BS_OFF + s B
constexpr u32 TC_SMEM_BYTES = TC_BAR_OFF + 128;                    // + 12 mbarriers, TMEM address, abort flag
constexpr long long TC_SPIN_LIMIT = 1ll << 22;                     // bounded mbarrier waits

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

// Waits for phase `parity` of the mbarrier at shared address bar, for at most `limit` polls.
// Gives up at once when *abort_flag is set (another role gave up) and, when the limit runs out,
// sets *abort_flag (so that every role leaves) and, if err is not null, *err.
__device__ __forceinline__ bool mbar_wait_bounded(u32 bar, u32 parity, long long limit, volatile int* abort_flag,
                                                  int* err) {
    for (long long it = 0; it < limit; it++) {
        if (*abort_flag) return false;
        u32 ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    *abort_flag = 1;
    if (err) atomicExch(err, 1);
    return false;
}

// Failure-detection self-test: one CTA waits on an mbarrier that nothing arrives at, through the
// tensor-core MAC's bounded wait, which must give up and report through *err.
__global__ void k_wait_selftest(int* err, long long limit) {
    __shared__ __align__(8) u64 bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    mbar_wait_bounded(smem_u32(&bar), 0, limit, &abort_flag, err);
}

// byte offset of element (row, kk) inside a K-major no-swizzle tile with 64-term rows
__device__ __forceinline__ u32 kmajor_off(u32 row, u32 kk) {
    return (row >> 3) * TC_SBO + (kk >> 3) * 128u + (row & 7u) * 16u + (kk & 7u) * 2u;
}

__device__ __forceinline__ u64 smem_desc(u32 saddr) {
    u64 d = 0;
    d |= (u64)((saddr & 0x3FFFFu) >> 4);          // start address
    d |= (u64)(128u >> 4) << 16;                   // leading byte offset (K direction)
    d |= (u64)(TC_SBO >> 4) << 32;                 // stride byte offset (M/N direction)
    d |= (u64)1 << 46;                             // fixed 0b001 at bits 46-48
    return d;                                      // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D f32, A and B f16, both K-major, N>>3 at 17, M>>4 at 24
__host__ __device__ constexpr u32 tc_idesc(u32 M, u32 N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}


// Persistent: each CTA walks work items blockIdx.x, blockIdx.x + gridDim.x, ... of every layer
// of the table; an item is ((row unit, polynomial, limb), slot tile, row tile) of one layer.
// The (item, K tile) pairs of a CTA form one stream with global index g: raw slot g % TC_RAW,
// MMA stage g % 2.  Warp 0 issues the bulk copies two stream positions ahead, across item
// boundaries, so the next item's rows load while the current item's epilogue runs.
struct TcItem {
    const LayerDev* ly;
    u32 ru, p, k, n0, row0, nrows, n_tiles;
};

// With clusters of CL CTAs (operand-image MAC), an item is (row unit, polynomial, limb, slot
// tile, group of CL row tiles) and CTA `rank` of the cluster takes row tile group * CL + rank.
template <int MAXB>
__device__ __forceinline__ bool tc_item(const Batch<MAXB>& B, u32 item, u32 N, u32 L, TcItem& it, u32 rank = 0,
                                        u32 CL = 1) {
    if (item >= B.start[ST_MAC][B.n]) return false;
    const u32 li = find_layer(B, ST_MAC, item);
    const LayerDev& Ly = B.L[li];
    const u32 rpc = Ly.tc_rows_per_cta, mtiles = (Ly.tc_rows + rpc - 1) / rpc, nt_n = N / TC_MTILE;
    const u32 mgroups = mtiles / CL;
    const u32 local = item - B.start[ST_MAC][li];
    const u32 mt = (local % mgroups) * CL + rank, nt = (local / mgroups) % nt_n, z = local / (mgroups * nt_n);
    it.ly = &Ly;
    it.k = z % L, it.p = (z / L) & 1, it.ru = z / (2 * L);
    it.n0 = nt * TC_MTILE;
    it.row0 = mt * rpc;
    it.nrows = min(rpc, Ly.tc_rows - it.row0);
    it.n_tiles = Ly.Kpad / TC_KTILE;
    return true;
}

// The work items of one CTA (or cluster) of the operand-image MAC, in order.  With clusters the items
// of the launch go round-robin over the clusters.  Without, the items of each layer run in rounds of
// G = floor(n_cl / R) R CTAs, R the layer's row tiles: the R row tiles of a slot tile (consecutive
// items) then always run in the same round, on CTAs that ran one slot tile's tiles together in the
// round before, so they stream the same images at about the same time and the later readers find
// them in L2 (with G = n_cl a team would straddle rounds whenever R does not divide n_cl, and its
// members would read the images an item apart, from DRAM).
struct TcWalk {
    u32 li, local, item;
};
template <int MAXB>
__device__ __forceinline__ bool tc_walk(const Batch<MAXB>& B, u32 cid, u32 n_cl, u32 N, u32 L, TcWalk& w, bool first,
                                        TcItem& it, u32 rank, u32 CL) {
    if (CL > 1) {
        w.item = first ? cid : w.item + n_cl;
        return tc_item(B, w.item, N, L, it, rank, CL);
    }
    auto rounds = [&](u32 li) {
        const LayerDev& Ly = B.L[li];
        const u32 R = max(1u, (Ly.tc_rows + Ly.tc_rows_per_cta - 1) / Ly.tc_rows_per_cta);
        return n_cl >= R ? n_cl / R * R : n_cl;
    };
    if (first) w.li = 0, w.local = cid;
    else w.local += rounds(w.li);
    for (; w.li < B.n; w.li++, w.local = cid) {
        if (cid < rounds(w.li) && w.local < B.start[ST_MAC][w.li + 1] - B.start[ST_MAC][w.li])
            return tc_item(B, B.start[ST_MAC][w.li] + w.local, N, L, it, 0, 1);
    }
    return false;
}

// Warp roles: warp 0 issues the copies, warp 1 (lane 0) issues the MMAs, warps 2..15 convert
// residues to fp16 chunks, warps 4..15 also run the epilogue.  Barriers (all bounded waits):
//   raw_full[s]   copies of stream position g landed in slot s = g % TC_RAW   (1 arrive + tx)
//   raw_empty[s]  slot s read by every converter warp and by the MMAs          (TC_CONV + 1)
//   a_full[st]    converted stage st = g % 2 written by every converter warp   (TC_CONV)
//   a_empty[st]   MMAs of stage st done                                          (1, commit)
//   acc_full      last MMA of a work item done                                   (1, commit)
//   acc_empty     accumulators read by every epilogue warp                       (TC_EPI)
constexpr int TC_CONV = TC_THREADS / 32 - 2;  // converter warps 2..15
constexpr int TC_EPI = TC_THREADS / 32 - 4;   // epilogue warps 4..15
static_assert(TC_THREADS == 512, "warp roles assume 16 warps");

template <bool PACKED, int MAXB>
__global__ void __launch_bounds__(TC_THREADS, 1) k_mac_tc(const __grid_constant__ Batch<MAXB> B, KP kp, u32 tmem_cols) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    constexpr int NR = PACKED ? 2 : 1;
    const u32 N = kp.N, L = kp.L;
    const u32 tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    u64* bars = reinterpret_cast<u64*>(tsm + TC_BAR_OFF);
    // barrier indices: raw_full 0..2, raw_empty 3..5, a_full 6..7, a_empty 8..9, acc_full 10, acc_empty 11
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    u32* tmem_slot = reinterpret_cast<u32*>(tsm + TC_BAR_OFF + 12 * 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tsm + TC_BAR_OFF + 12 * 8 + 4);

    if (tid == 0) {
        const u32 counts[12] = {1, 1, 1, TC_CONV + 1, TC_CONV + 1, TC_CONV + 1, TC_CONV, TC_CONV, 1, 1, 1, TC_EPI};
        for (int i = 0; i < 12; i++) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(i)), "r"(counts[i]));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const u32 tmem = *tmem_slot;

    // bounded wait that gives up at once when another role has given up; an abort leaves the
    // CTA's remaining items of every layer of the table unfinished, so the drain below marks the
    // status word of every layer
    auto wait = [&](int i, u32 parity) -> bool {
        return mbar_wait_bounded(bar(i), parity, TC_SPIN_LIMIT, abort_flag, nullptr);
    };
    auto arrive = [&](int i) { asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(i)) : "memory"); };

    if (warp == 0) {
        // ---------------------------------------------------------------- copies
        u32 g = 0;
        TcItem it;
        for (u32 item = blockIdx.x; tc_item(B, item, N, L, it); item += gridDim.x) {
            const LayerDev& Ly = *it.ly;
            const u32 bbytes = Ly.tc_rows_per_cta * TC_KTILE * 2, ktiles = Ly.Kpad / TC_KTILE;
            const u32 mt = it.row0 / Ly.tc_rows_per_cta;
            for (u32 t = 0; t < it.n_tiles; t++, g++) {
                const u32 s = g % TC_RAW;
                const bool fr = g < TC_RAW || wait(3 + s, ((g / TC_RAW) - 1) & 1);
                if (!__all_sync(0xffffffffu, fr)) break;
                if (lane == 0) {
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(s)),
                                 "r"(TC_RAW_BYTES + bbytes)
                                 : "memory");
                    const int x = (int)it.n0, y = (int)(it.p * L + it.k);
                    const int z = (int)(it.ru * Ly.in_groups * Ly.n_rot + t * TC_KTILE);
                    asm volatile(
                        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
                            "r"(smem_u32(tsm + TC_RAW_OFF + s * TC_RAW_BYTES)),
                        "l"(reinterpret_cast<u64>(&Ly.rmap)), "r"(x), "r"(y), "r"(z), "r"(bar(s))
                        : "memory");
                    const __half* bsrc = Ly.sc16 + ((size_t)mt * ktiles + t) * (Ly.tc_rows_per_cta * TC_KTILE);
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(tsm + TC_BS_OFF + s * TC_B_BYTES)),
                        "l"(bsrc), "r"(bbytes), "r"(bar(s))
                        : "memory");
                }
                __syncwarp();
            }
            if (*abort_flag) break;
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMAs (lane 0)
        if (lane == 0) {
            u32 g = 0, unit = 0;  // unit = (item, segment): one accumulation in TMEM
            TcItem it;
            for (u32 item = blockIdx.x; tc_item(B, item, N, L, it); item += gridDim.x) {
                const u32 idesc = tc_idesc(TC_MTILE, it.nrows);
                bool okk = true;
                for (u32 t = 0; t < it.n_tiles; t++, g++) {
                    const u32 st = g & 1, s = g % TC_RAW, tseg = t % TC_SEG_TILES;
                    if (tseg == 0) {
                        if (unit > 0 && !wait(11, (unit - 1) & 1)) { okk = false; break; }  // accumulators read out
                        asm volatile("tcgen05.fence::after_thread_sync;");
                    }
                    if (!wait(6 + st, (g >> 1) & 1)) { okk = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const u32 a_base = smem_u32(tsm + st * TC_STAGE_BYTES), b_base = smem_u32(tsm + TC_BS_OFF + s * TC_B_BYTES);
#pragma unroll
                    for (int c = 0; c < TC_CHUNKS; c++) {
#pragma unroll
                        for (int ks = 0; ks < TC_KTILE / 16; ks++) {
                            const u64 ad = smem_desc(a_base + c * TC_A_CHUNK_BYTES + ks * 256);
                            const u64 bd = smem_desc(b_base + ks * 256);
                            const u32 acc = (tseg > 0 || ks > 0) ? 1u : 0u;
                            const u32 dt = tmem + (u32)(c * it.nrows);
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar(8 + st)));
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar(3 + s)));
                    if (tseg == TC_SEG_TILES - 1 || t + 1 == it.n_tiles) {
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar(10)));
                        unit++;
                    }
                }
                if (!okk) break;
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- converters (+ epilogue)
        u32 g = 0, unit = 0;
        TcItem it;
        const u32 cw = warp - 2;  // converter index 0..13
        for (u32 item = blockIdx.x; tc_item(B, item, N, L, it); item += gridDim.x) {
            const LayerDev& Ly = *it.ly;
            const u32 K = Ly.K;
            bool okk = true;
            for (u32 t = 0; t < it.n_tiles; t++, g++) {
                const u32 st = g & 1, s = g % TC_RAW, kk0 = t * TC_KTILE;
                bool w = wait(s, (g / TC_RAW) & 1);                    // raw data landed
                w = w && (g < 2 || wait(8 + st, ((g >> 1) - 1) & 1));  // stage free
                if (!__all_sync(0xffffffffu, w)) { okk = false; break; }
                const u64* raw = reinterpret_cast<const u64*>(tsm + TC_RAW_OFF + s * TC_RAW_BYTES);
                unsigned char* A = tsm + st * TC_STAGE_BYTES;
                // 512 (slot, octet) pieces per tile over 14 warps: piece i = slot (i % 128), octet (i / 128)
                for (u32 i = cw * 32 + lane; i < TC_MTILE * (TC_KTILE / 8); i += TC_CONV * 32) {
                    const u32 nl = i & (TC_MTILE - 1), o = i >> 7;
                    u64 v[8];
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const u32 r = o * 8 + e;
                        v[e] = (kk0 + r < K) ? raw[r * TC_MTILE + nl] : 0;
                    }
                    // the five 10-bit chunks of each residue as the low bits of 32-bit words, taken
                    // from its 32-bit halves (chunk 3 straddles them: a funnel shift)
                    u32 cw8[TC_CHUNKS][8];
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const u32 lo = (u32)v[e], hi = (u32)(v[e] >> 32);
                        cw8[0][e] = lo;
                        cw8[1][e] = lo >> 10;
                        cw8[2][e] = lo >> 20;
                        cw8[3][e] = __funnelshift_r(lo, hi, 30);
                        cw8[4][e] = hi >> 8;
                    }
#pragma unroll
                    for (int c = 0; c < TC_CHUNKS; c++) {
                        u32 w[4];
#pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            // fp16 bits of 1024 + x are 0x6400 | x; subtracting 1536 gives x - 512 exactly
                            const u32 packed = (cw8[c][e] & 0x3FFu) | ((cw8[c][e + 1] << 16) & 0x3FF0000u) | 0x64006400u;
                            __half2 h = *reinterpret_cast<const __half2*>(&packed);
                            h = __hsub2(h, __float2half2_rn(1536.0f));
                            w[e / 2] = *reinterpret_cast<u32*>(&h);
                        }
                        *reinterpret_cast<uint4*>(A + c * TC_A_CHUNK_BYTES + kmajor_off(nl, o * 8)) =
                            make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    arrive(6 + st);  // stage written
                    arrive(3 + s);   // raw slot read
                }
                if (warp < 4 || (t % TC_SEG_TILES != TC_SEG_TILES - 1 && t + 1 != it.n_tiles)) continue;
                // epilogue of segment seg: warp w reads TMEM lanes 32 (w % 4) + lane; the three
                // warps of a sub-partition take every third 8-column block of output rows
                const u32 seg = t / TC_SEG_TILES;
                if (!__all_sync(0xffffffffu, wait(10, unit & 1))) { okk = false; break; }
                unit++;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const u32 sp = warp & 3, third = (warp - 4) >> 2;
                const u32 nl = sp * 32 + lane, x = it.n0 + nl, nrows = it.nrows, row0 = it.row0, k = it.k, p = it.p;
                const LimbC m = kp.limb[k];
                const u64 pkv = PACKED ? Ly.pk[(size_t)k * N + x] : 0, pksv = PACKED ? Ly.pksh[(size_t)k * N + x] : 0;
                for (u32 cb = third * 8; cb < nrows; cb += 24) {
                    u32 d[TC_CHUNKS][8];
#pragma unroll
                    for (int c = 0; c < TC_CHUNKS; c++) {
                        const u32 ta = tmem + ((sp * 32u) << 16) + (u32)(c * nrows) + cb;
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                     : "=r"(d[c][0]), "=r"(d[c][1]), "=r"(d[c][2]), "=r"(d[c][3]), "=r"(d[c][4]),
                                       "=r"(d[c][5]), "=r"(d[c][6]), "=r"(d[c][7])
                                     : "r"(ta));
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    u64 red[8];
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const long long b = Ly.bias[(size_t)seg * Ly.tc_rows + row0 + cb + j];  // 512 S of the segment
                        const long long lo = ((long long)__float2int_rn(__uint_as_float(d[0][j])) + b) +
                                             (((long long)__float2int_rn(__uint_as_float(d[1][j])) + b) << 10) +
                                             (((long long)__float2int_rn(__uint_as_float(d[2][j])) + b) << 20);
                        const long long hi = ((long long)__float2int_rn(__uint_as_float(d[3][j])) + b) +
                                             (((long long)__float2int_rn(__uint_as_float(d[4][j])) + b) << 10);
                        red[j] = tc_reduce(lo, hi, m);
                    }
#pragma unroll
                    for (int j = 0; j < 8; j += NR) {
                        const u32 row = row0 + cb + j;
                        const u32 gg = row / NR;
                        if (gg >= Ly.out_groups) continue;
                        u64 out = red[j];
                        if (PACKED) out = addq(mulmod_shoup(out, kp.kmul, m.ksh, m.q), mulmod_shoup(red[j + 1], pkv, pksv, m.q), m.q);
                        u64* o = Ly.O + ((size_t)(it.ru * Ly.out_groups + gg) * 2 + p) * L * N + (size_t)k * N + x;
                        if (seg > 0) out = addq(out, *o, m.q);  // this thread stored the earlier segments
                        *o = out;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) arrive(11);  // accumulators free
            }
            if (!okk) break;
        }
    }
    // drain: every copy that was issued is waited for by the converters in the normal path; after an
    // abort, give in-flight copies and MMAs a bounded time to land before TMEM is freed
    // (after every role has left its loop, so that a wait that gave up late is still reported)
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (*abort_flag && tid == 0) {
        for (u32 i = 0; i < B.n; i++) atomicExch(B.L[i].err, 1);
        for (long long i = 0; i < TC_SPIN_LIMIT / 16; i++) __nanosleep(64);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
}

// ------------------------------------------------------------------ operand-image form
// The key switch writes the rotated residues straight into the shared-memory image the
// tensor-core MMA reads (five fp16 chunks per residue, K-major core matrices), so the MAC is
// a pure copy -> MMA pipeline and a residue is split into chunks once, not once per row tile.
//
// Term order of the image form: kk = rot * in_pad + j (rotation-major; in_pad = in_groups
// rounded up to 8, the padded terms carry zero scalars), so eight consecutive terms of one
// slot are eight input ciphertexts of one rotation: one 16-byte store per chunk.
// Image of (row unit, polynomial, limb, slot tile nt, K tile kt): 5 chunks x 8 KB, chunk c at
// byte c * 8192, element (slot row m, term kl) at (m >> 3) * 512 + (kl >> 3) * 128 + (m & 7) * 16
// + (kl & 7) * 2, the layout smem_desc describes (LBO 128 B, SBO 512 B).
constexpr u32 KSI_JB = 8;                 // input ciphertexts per block (one group of eight)
constexpr u32 IMG_HALVES = TC_CHUNKS * TC_MTILE * TC_KTILE;  // 20480 halves = 40 KB per image

// Step 2, operand-image form.  Local block = (row unit and group of eight input ciphertexts,
// rotation group, source slot tile nt, limb k), the (row unit, group) pair varying fastest so
// that consecutive blocks read the same key tiles.  The block keeps the digit transforms of its
// eight ciphertexts (tile nt, limb k) in shared memory and runs every rotation of its group over
// them: a digit transform is read from memory once, not once per rotation.  Thread (slot, half)
// owns the SOURCE slot y = nt * 128 + slot (coalesced loads) and four of the eight ciphertexts;
// for rotation r it produces the destination x = src_r^-1(y), which lies in one aligned
// destination tile xt_r for the whole block (sigma maps aligned tiles onto aligned tiles).  The
// key words of rotation r + 1 are copied into shared memory (cp.async) while rotation r is
// computed.  The chunks of the eight ciphertexts gather in a shared copy of the destination
// tile's image rows (row x & 127), which leave in 16-byte pieces.  Small layers split their
// rotations into groups so that the grid still fills the GPU.
constexpr int KSI_THREADS = 256;          // 128 source slots x 2 halves of the eight ciphertexts
constexpr int KSI_JH = 4;                 // input ciphertexts per thread
constexpr u32 KSI_TARGET_BLOCKS = 1024;   // rotation groups raise a layer's grid up to about this

// rows [2][5][128] uint4, digit transforms [8][LL][128] u64, key words [2 buffers][2][LL][128] u64
__host__ __device__ constexpr size_t ksi_smem_bytes(u32 LL) {
    return (size_t)2 * TC_CHUNKS * TC_MTILE * 16 + ((size_t)KSI_JB * LL + 4 * LL) * TC_MTILE * 8;
}

// rotation groups of the image key switch: as few as give about KSI_TARGET_BLOCKS blocks, each of
// ceil(n_rot_all / groups) rotations, and none empty (9 rotations in 4 groups of 3 would leave the
// fourth without a rotation: they become 3 groups)
__host__ __device__ inline u32 ksi_groups(u32 row_units, u32 in_pad, u32 n_rot_all, u32 L, u32 N) {
    const u64 base = (u64)row_units * ((in_pad + KSI_JB - 1) / KSI_JB) * L * (N / TC_MTILE);
    u64 g = (KSI_TARGET_BLOCKS + base - 1) / base;
    g = g < 1 ? 1 : (g > n_rot_all ? n_rot_all : g);
    const u64 per = (n_rot_all + g - 1) / g;
    return (u32)((n_rot_all + per - 1) / per);
}

__device__ __forceinline__ uint2 chunk_pack4(const u64 (&v)[KSI_JH], int c) {
    u32 w[2];
#pragma unroll
    for (int e = 0; e < KSI_JH; e += 2) {
        u32 a, b;
        const u32 la = (u32)v[e], ha = (u32)(v[e] >> 32), lb = (u32)v[e + 1], hb = (u32)(v[e + 1] >> 32);
        switch (c) {
            case 0: a = la, b = lb; break;
            case 1: a = la >> 10, b = lb >> 10; break;
            case 2: a = la >> 20, b = lb >> 20; break;
            case 3: a = __funnelshift_r(la, ha, 30), b = __funnelshift_r(lb, hb, 30); break;
            default: a = ha >> 8, b = hb >> 8; break;
        }
        // fp16 bits of 1024 + x are 0x6400 | x (x < 1024); subtracting 1536 gives x - 512 exactly
        const u32 packed = (a & 0x3FFu) | ((b << 16) & 0x3FF0000u) | 0x64006400u;
        __half2 h = *reinterpret_cast<const __half2*>(&packed);
        h = __hsub2(h, __float2half2_rn(1536.0f));
        w[e / 2] = *reinterpret_cast<u32*>(&h);
    }
    return make_uint2(w[0], w[1]);
}

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int LL, int MAXB>
__global__ void __launch_bounds__(KSI_THREADS, LL <= 4 ? 3 : (LL <= 8 ? 2 : 1)) k_keyswitch_img(const __grid_constant__ Batch<MAXB> B, KP kp) {
    extern __shared__ __align__(16) unsigned char ksm[];
    uint4 (*rows)[TC_CHUNKS][TC_MTILE] = reinterpret_cast<uint4 (*)[TC_CHUNKS][TC_MTILE]>(ksm);
    u64* const Dsm = reinterpret_cast<u64*>(ksm + 2 * TC_CHUNKS * TC_MTILE * 16);
    u64* const Ksm = Dsm + KSI_JB * LL * TC_MTILE;
    const u32 li = find_layer(B, ST_KS, blockIdx.x);
    const LayerDev& Ly = B.L[li];
    const u32 N = kp.N, L = kp.L, logN = kp.logN, NT = N / TC_MTILE;
    const u32 JC = (Ly.in_pad + KSI_JB - 1) / KSI_JB, QJ = Ly.row_units * JC, RG = Ly.ks_rg;
    u32 local = blockIdx.x - B.start[ST_KS][li];
    const u32 q = local % QJ;
    local /= QJ;
    const u32 g = local % RG;
    local /= RG;
    const u32 nt = local % NT, k = local / NT;
    const u32 ru = q / JC, jc = q % JC;
    const u32 tid = threadIdx.x, slot = tid & (TC_MTILE - 1), h = tid / TC_MTILE;
    const u32 src = nt * TC_MTILE + slot;
    const LimbC m = kp.limb[k];
    const u32 rpg = (Ly.n_rot_all + RG - 1) / RG, r_begin = g * rpg, r_end = min(Ly.n_rot_all, r_begin + rpg);
    const u32 j0 = jc * KSI_JB, ja = h * KSI_JH;  // the block's first ciphertext; this thread's within the eight
    const u32 nj = j0 >= Ly.in_groups ? 0u : min(KSI_JB, Ly.in_groups - j0);  // real terms; the rest are padding
    const size_t ctw = 2ull * L * N, d_step = (size_t)LL * L * N, dd_step = (size_t)L * N;
    const size_t r_step = (size_t)Ly.r_slots * ctw;
    const u32 ktiles = Ly.Kpad / TC_KTILE;
    const u32 e_src = 2 * (__brev(src) >> (32 - logN)) + 1;
    const u32 row_off = (slot >> 3) * 256 + (slot & 7) * 8;  // halves: image row `slot` within a chunk
    // this thread's four ciphertexts: c0 in registers, the digit transforms in shared memory (read
    // back by this thread only, so no barrier is needed before their use)
    const size_t c_first = (size_t)ru * Ly.in_groups + j0 + ja;
    const u64* const Rp = Ly.R + (c_first * Ly.r_slots + Ly.r_id) * ctw + (size_t)k * N + src;
    u64 c0[KSI_JH];
#pragma unroll
    for (int jj = 0; jj < KSI_JH; jj++) {
        const bool real = ja + jj < nj;
        c0[jj] = real ? __ldg(Rp + jj * r_step) : 0;
        const u64* Dc = Ly.D + (c_first + jj) * d_step + (size_t)k * N + src;
#pragma unroll
        for (int dd = 0; dd < LL; dd++) Dsm[((ja + jj) * LL + dd) * TC_MTILE + slot] = real ? __ldg(Dc + dd * dd_step) : 0;
    }
    auto dest = [&](u32 galois_inv) {
        const u32 e2 = (u32)(((u64)e_src * galois_inv) & (2ull * N - 1));
        return __brev((e2 - 1) >> 1) >> (32 - logN);
    };
    // key words of rotation r at this thread's destination, polynomial h, every digit -> buffer b
    auto fetch_keys = [&](u32 r, u32 b) {
        const RotDev rd = Ly.rots_all[r];
        if (r == Ly.id_rot) return;
        const u64* kb = Ly.ksk + (size_t)rd.key * LL * 2 * L * N + ((size_t)h * L + k) * N + dest(rd.galois_inv);
#pragma unroll
        for (int dd = 0; dd < LL; dd++)
            cp_async8(&Ksm[((b * 2 + h) * LL + dd) * TC_MTILE + slot], kb + (size_t)dd * 2 * L * N);
        cp_async_commit();
    };
    const int kind = m.sm1 == 49 ? (m.delta ? 1 : 2) : 3;
    if (r_begin < r_end) fetch_keys(r_begin, 0);  // (ksi_groups leaves no group empty)
    cp_async_wait_all();
    __syncthreads();
#pragma unroll 1
    for (u32 r = r_begin; r < r_end; r++) {
        const u32 b = (r - r_begin) & 1;
        if (r + 1 < r_end) fetch_keys(r + 1, b ^ 1);
        const RotDev rd = Ly.rots_all[r];
        const u32 x = dest(rd.galois_inv), xl = x & (TC_MTILE - 1), xt = x / TC_MTILE;
        u64 v0[KSI_JH], v1[KSI_JH];
        if (r == Ly.id_rot) {
            // the identity converts NTT(c0), NTT(c1) as they are
#pragma unroll
            for (int jj = 0; jj < KSI_JH; jj++) {
                v0[jj] = c0[jj];
                v1[jj] = ja + jj < nj ? __ldg(Rp + jj * r_step + dd_step) : 0;
            }
        } else {
            // keys of the destination x split at bit 25 (see k_keyswitch), for the four ciphertexts
            u32 k0l[LL], k0h[LL], k1l[LL], k1h[LL];
            const u64* K0 = Ksm + (size_t)(b * 2 + 0) * LL * TC_MTILE + slot;
            const u64* K1 = Ksm + (size_t)(b * 2 + 1) * LL * TC_MTILE + slot;
#pragma unroll
            for (int dd = 0; dd < LL; dd++) {
                const u64 a = K0[dd * TC_MTILE], bb = K1[dd * TC_MTILE];
                k0l[dd] = (u32)(a & 0x1FFFFFFu), k0h[dd] = (u32)(a >> 25);
                k1l[dd] = (u32)(bb & 0x1FFFFFFu), k1h[dd] = (u32)(bb >> 25);
            }
            if (kind <= 2) {
                // 50-bit limbs: Karatsuba middle term, one reduction per sum (see k_keyswitch)
                u32 k0s[LL], k1s[LL];
#pragma unroll
                for (int dd = 0; dd < LL; dd++) k0s[dd] = k0l[dd] + k0h[dd], k1s[dd] = k1l[dd] + k1h[dd];
#pragma unroll
                for (int jj = 0; jj < KSI_JH; jj++) {
                    v0[jj] = v1[jj] = 0;
                    if (ja + jj >= nj) continue;
                    const u64* Dc = Dsm + (size_t)(ja + jj) * LL * TC_MTILE + slot;
                    u64 lo0 = 0, mid0 = 0, hi0 = 0, lo1 = 0, mid1 = 0, hi1 = 0;
#pragma unroll
                    for (int dd = 0; dd < LL; dd++) {
                        const u64 dv = Dc[dd * TC_MTILE];
                        const u32 dl = (u32)dv, dh = (u32)(dv >> 32), ds = dl + dh;  // stored split at bit 25
                        mad_wide_u(lo0, dl, k0l[dd]);
                        mad_wide_u(hi0, dh, k0h[dd]);
                        mad_wide_u(mid0, ds, k0s[dd]);
                        mad_wide_u(lo1, dl, k1l[dd]);
                        mad_wide_u(hi1, dh, k1h[dd]);
                        mad_wide_u(mid1, ds, k1s[dd]);
                    }
                    mid0 -= lo0 + hi0;
                    mid1 -= lo1 + hi1;
                    lo0 += c0[jj];  // + sigma(c0)
                    if (kind == 1) {
                        v0[jj] = fold_reduce50(lo0, mid0, hi0, m);
                        v1[jj] = fold_reduce50(lo1, mid1, hi1, m);
                    } else {
                        v0[jj] = bred_split50(lo0, mid0, hi0, m);
                        v1[jj] = bred_split50(lo1, mid1, hi1, m);
                    }
                }
            } else {
#pragma unroll
                for (int jj = 0; jj < KSI_JH; jj++) {
                    v0[jj] = v1[jj] = 0;
                    if (ja + jj >= nj) continue;
                    const u64* Dc = Dsm + (size_t)(ja + jj) * LL * TC_MTILE + slot;
                    u64 lo0 = 0, mid0 = 0, hi0 = 0, lo1 = 0, mid1 = 0, hi1 = 0;
#pragma unroll
                    for (int dd = 0; dd < LL; dd++) {
                        const u64 dv = Dc[dd * TC_MTILE];
                        const u32 dl = (u32)dv, dh = (u32)(dv >> 32);  // stored split at bit 25
                        mad_wide_u(lo0, dl, k0l[dd]);
                        mad_wide_u(mid0, dl, k0h[dd]);
                        mad_wide_u(mid0, dh, k0l[dd]);
                        mad_wide_u(hi0, dh, k0h[dd]);
                        mad_wide_u(lo1, dl, k1l[dd]);
                        mad_wide_u(mid1, dl, k1h[dd]);
                        mad_wide_u(mid1, dh, k1l[dd]);
                        mad_wide_u(hi1, dh, k1h[dd]);
                    }
                    lo0 += c0[jj];
                    v0[jj] = bred128(((u128)hi0 << 50) + ((u128)mid0 << 25) + lo0, m);
                    v1[jj] = bred128(((u128)hi1 << 50) + ((u128)mid1 << 25) + lo1, m);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < TC_CHUNKS; c++) {
            reinterpret_cast<uint2*>(&rows[0][c][xl])[h] = chunk_pack4(v0, c);
            reinterpret_cast<uint2*>(&rows[1][c][xl])[h] = chunk_pack4(v1, c);
        }
        __syncthreads();
        {
            // thread (slot, p = h) writes image row `slot` of polynomial h: terms r in_pad + j0 .. + 7
            const u32 kk = r * Ly.in_pad + j0, kt = kk / TC_KTILE, kl = kk % TC_KTILE;
            __half* d0 = Ly.A16 + ((((size_t)ru * 2 + h) * L + k) * NT + xt) * ktiles * IMG_HALVES +
                         (size_t)kt * IMG_HALVES + (kl >> 3) * 64 + row_off;
#pragma unroll
            for (int c = 0; c < TC_CHUNKS; c++)
                __stcs(reinterpret_cast<uint4*>(d0 + c * (TC_MTILE * TC_KTILE)), rows[h][c][slot]);
        }
        cp_async_wait_all();  // the next rotation's keys, made visible to the other half by the barrier
        __syncthreads();
    }
    // the terms past n_rot in_pad that fill the last K tile carry zero scalars; their operands must
    // still be finite numbers (a NaN times 0 is NaN), so the blocks of the last ciphertext group and
    // rotation group zero them, each for the destination tile numbered as its source tile
    if (jc + 1 == JC && g + 1 == RG) {
        __half* d0 = Ly.A16 + ((((size_t)ru * 2 + h) * L + k) * NT + nt) * ktiles * IMG_HALVES + row_off;
        for (u32 kk = Ly.n_rot_all * Ly.in_pad; kk < Ly.Kpad; kk += 8) {
            const u32 kt = kk / TC_KTILE, kl = kk % TC_KTILE;
#pragma unroll
            for (int c = 0; c < TC_CHUNKS; c++)
                __stcs(reinterpret_cast<uint4*>(d0 + (size_t)kt * IMG_HALVES + (kl >> 3) * 64 + c * (TC_MTILE * TC_KTILE)),
                       make_uint4(0, 0, 0, 0));
        }
    }
}

// Step 3, operand-image form: the tensor-core contraction of k_mac_tc with the operands copied
// ready-made.  Warp 0 issues one bulk copy of the 40 KB image and one of the scalar tile per
// K tile into a ring of TCI_STAGES stages; warp 1 (lane 0) issues the MMAs; warps 4..15 run the
// epilogue of each accumulation segment (as in k_mac_tc).  Barriers (all bounded waits):
//   full[s]    image and scalars of stream position g landed in stage s = g % TCI_STAGES
//   empty[s]   MMAs of stage s done (commit)
//   acc_full   last MMA of an accumulation segment done (commit)
//   acc_empty  accumulators read by every epilogue warp
constexpr int TCI_STAGES = 4;
constexpr u32 TCI_A_BYTES = IMG_HALVES * 2;                       // 40 KB
constexpr u32 TCI_B_OFF = TCI_STAGES * TCI_A_BYTES;               // scalar tiles after the images
constexpr u32 TCI_BAR_OFF = TCI_B_OFF + TCI_STAGES * TC_B_BYTES;
constexpr u32 TCI_SMEM_BYTES = TCI_BAR_OFF + 128;                 // 2 TCI_STAGES + 2 mbarriers, TMEM slot, flag
static_assert(TCI_SMEM_BYTES <= 227 * 1024, "operand-image MAC exceeds shared memory");

// Clusters (CL = 2, 4, 8): the CL CTAs of a cluster take the row tiles of one slot tile and share
// each image: CTA `rank` copies bytes [rank, rank + 1) x 40 KB / CL of it with one multicast bulk
// copy into the same stage of every CTA of the cluster, and every CTA's MMA completion is
// committed to the `empty` barrier of every CTA, so no CTA refills a stage (in any CTA) before all
// have used it.  A cluster barrier at start (barrier initialisation) and at exit (no copy or
// commit may still target a CTA that has left) brackets the work.
template <bool PACKED, int CL, int MAXB>
__global__ void __launch_bounds__(TC_THREADS, 1) k_mac_img(const __grid_constant__ Batch<MAXB> B, KP kp, u32 tmem_cols) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    constexpr int NR = PACKED ? 2 : 1;
    constexpr int NB = 2 * TCI_STAGES + 2;
    const u32 N = kp.N, L = kp.L, NT = N / TC_MTILE;
    const u32 tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    u32 rank = 0;
    if (CL > 1) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const u32 cid = blockIdx.x / CL, n_cl = gridDim.x / CL;
    constexpr u32 SLICE = TCI_A_BYTES / CL;  // bytes of an image each CTA of a cluster copies
    const uint16_t cta_mask = (uint16_t)((1u << CL) - 1);
    u64* bars = reinterpret_cast<u64*>(tsm + TCI_BAR_OFF);
    // barrier indices: full 0..S-1, empty S..2S-1, acc_full 2S, acc_empty 2S+1
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    constexpr int FULL = 0, EMPTY = TCI_STAGES, ACC_FULL = 2 * TCI_STAGES, ACC_EMPTY = 2 * TCI_STAGES + 1;
    u32* tmem_slot = reinterpret_cast<u32*>(tsm + TCI_BAR_OFF + NB * 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tsm + TCI_BAR_OFF + NB * 8 + 4);

    if (tid == 0) {
        for (int i = 0; i < TCI_STAGES; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(FULL + i)), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(EMPTY + i)), "r"(CL));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(ACC_FULL)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(ACC_EMPTY)), "r"(TC_EPI));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    if (CL > 1) {
        // every CTA's barriers are initialised before any CTA of the cluster copies or commits to them
        asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    const u32 tmem = *tmem_slot;

    auto wait = [&](int i, u32 parity) -> bool {
        return mbar_wait_bounded(bar(i), parity, TC_SPIN_LIMIT, abort_flag, nullptr);
    };
    auto arrive = [&](int i) { asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(i)) : "memory"); };

    if (warp == 0) {
        // ---------------------------------------------------------------- copies
        u32 g = 0;
        TcItem it;
        bool ok = true;
        TcWalk wk;
        for (bool f = true; ok && tc_walk(B, cid, n_cl, N, L, wk, f, it, rank, CL); f = false) {
            const LayerDev& Ly = *it.ly;
            const u32 bbytes = Ly.tc_rows_per_cta * TC_KTILE * 2, ktiles = Ly.Kpad / TC_KTILE;
            const u32 mt = it.row0 / Ly.tc_rows_per_cta, nt = it.n0 / TC_MTILE;
            const __half* abase = Ly.A16 + ((((size_t)it.ru * 2 + it.p) * L + it.k) * NT + nt) * ktiles * IMG_HALVES;
            for (u32 t = 0; t < it.n_tiles; t++, g++) {
                const u32 s = g % TCI_STAGES;
                const bool fr = g < TCI_STAGES || wait(EMPTY + s, ((g / TCI_STAGES) - 1) & 1);
                if (!__all_sync(0xffffffffu, fr)) { ok = false; break; }
                if (lane == 0) {
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(FULL + s)),
                                 "r"(TCI_A_BYTES + bbytes)
                                 : "memory");
                    if (CL == 1) {
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                smem_u32(tsm + s * TCI_A_BYTES)),
                            "l"(abase + (size_t)t * IMG_HALVES), "r"(TCI_A_BYTES), "r"(bar(FULL + s))
                            : "memory");
                    } else {
                        // this CTA's slice of the image, into the same stage of every CTA of the cluster
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
                            " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(tsm + s * TCI_A_BYTES + rank * SLICE)),
                            "l"(reinterpret_cast<const unsigned char*>(abase + (size_t)t * IMG_HALVES) + rank * SLICE),
                            "r"(SLICE), "r"(bar(FULL + s)), "h"(cta_mask)
                            : "memory");
                    }
                    const __half* bsrc = Ly.sc16 + ((size_t)mt * ktiles + t) * (Ly.tc_rows_per_cta * TC_KTILE);
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(tsm + TCI_B_OFF + s * TC_B_BYTES)),
                        "l"(bsrc), "r"(bbytes), "r"(bar(FULL + s))
                        : "memory");
                }
                __syncwarp();
            }
            if (*abort_flag) ok = false;
        }
        // with clusters, the other CTAs' MMAs commit to this CTA's empty barriers: wait for the
        // commits of the last uses of every stage, so none is still on its way when this CTA leaves
        if (CL > 1 && ok) {
            for (u32 gg = g > TCI_STAGES ? g - TCI_STAGES : 0; gg < g; gg++)
                if (!__all_sync(0xffffffffu, wait(EMPTY + gg % TCI_STAGES, (gg / TCI_STAGES) & 1))) break;
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMAs (lane 0)
        if (lane == 0) {
            u32 g = 0, unit = 0;  // unit = (item, segment): one accumulation in TMEM
            TcItem it;
            TcWalk wk;
            for (bool f = true; tc_walk(B, cid, n_cl, N, L, wk, f, it, rank, CL); f = false) {
                const u32 idesc = tc_idesc(TC_MTILE, it.nrows);
                bool okk = true;
                for (u32 t = 0; t < it.n_tiles; t++, g++) {
                    const u32 s = g % TCI_STAGES, tseg = t % TC_SEG_TILES;
                    if (tseg == 0) {
                        if (unit > 0 && !wait(ACC_EMPTY, (unit - 1) & 1)) { okk = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                    }
                    if (!wait(FULL + s, (g / TCI_STAGES) & 1)) { okk = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const u32 a_base = smem_u32(tsm + s * TCI_A_BYTES), b_base = smem_u32(tsm + TCI_B_OFF + s * TC_B_BYTES);
#pragma unroll
                    for (int c = 0; c < TC_CHUNKS; c++) {
#pragma unroll
                        for (int ks = 0; ks < TC_KTILE / 16; ks++) {
                            const u64 ad = smem_desc(a_base + c * TC_A_CHUNK_BYTES + ks * 256);
                            const u64 bd = smem_desc(b_base + ks * 256);
                            const u32 acc = (tseg > 0 || ks > 0) ? 1u : 0u;
                            const u32 dt = tmem + (u32)(c * it.nrows);
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                        }
                    }
                    if (CL == 1)
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            bar(EMPTY + s)));
                    else
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
                            " [%0], %1;" ::"r"(bar(EMPTY + s)),
                            "h"(cta_mask));
                    if (tseg == TC_SEG_TILES - 1 || t + 1 == it.n_tiles) {
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar(ACC_FULL)));
                        unit++;
                    }
                }
                if (!okk) break;
            }
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ---------------------------------------------------------------- epilogue
        u32 unit = 0;
        TcItem it;
        TcWalk wk;
        for (bool f = true; tc_walk(B, cid, n_cl, N, L, wk, f, it, rank, CL); f = false) {
            const LayerDev& Ly = *it.ly;
            const u32 n_seg = (it.n_tiles + TC_SEG_TILES - 1) / TC_SEG_TILES;
            bool okk = true;
            for (u32 seg = 0; seg < n_seg; seg++) {
                if (!__all_sync(0xffffffffu, wait(ACC_FULL, unit & 1))) { okk = false; break; }
                unit++;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const u32 sp = warp & 3, third = (warp - 4) >> 2;
                const u32 nl = sp * 32 + lane, x = it.n0 + nl, nrows = it.nrows, row0 = it.row0, k = it.k, p = it.p;
                const LimbC m = kp.limb[k];
                const u64 pkv = PACKED ? Ly.pk[(size_t)k * N + x] : 0, pksv = PACKED ? Ly.pksh[(size_t)k * N + x] : 0;
                for (u32 cb = third * 8; cb < nrows; cb += 24) {
                    u32 d[TC_CHUNKS][8];
#pragma unroll
                    for (int c = 0; c < TC_CHUNKS; c++) {
                        const u32 ta = tmem + ((sp * 32u) << 16) + (u32)(c * nrows) + cb;
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                     : "=r"(d[c][0]), "=r"(d[c][1]), "=r"(d[c][2]), "=r"(d[c][3]), "=r"(d[c][4]),
                                       "=r"(d[c][5]), "=r"(d[c][6]), "=r"(d[c][7])
                                     : "r"(ta));
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    u64 red[8];
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const long long b = Ly.bias[(size_t)seg * Ly.tc_rows + row0 + cb + j];  // 512 S of the segment
                        const long long lo = ((long long)__float2int_rn(__uint_as_float(d[0][j])) + b) +
                                             (((long long)__float2int_rn(__uint_as_float(d[1][j])) + b) << 10) +
                                             (((long long)__float2int_rn(__uint_as_float(d[2][j])) + b) << 20);
                        const long long hi = ((long long)__float2int_rn(__uint_as_float(d[3][j])) + b) +
                                             (((long long)__float2int_rn(__uint_as_float(d[4][j])) + b) << 10);
                        red[j] = tc_reduce(lo, hi, m);
                    }
#pragma unroll
                    for (int j = 0; j < 8; j += NR) {
                        const u32 row = row0 + cb + j;
                        const u32 gg = row / NR;
                        if (gg >= Ly.out_groups) continue;
                        u64 out = red[j];
                        if (PACKED) out = addq(mulmod_shoup(out, kp.kmul, m.ksh, m.q), mulmod_shoup(red[j + 1], pkv, pksv, m.q), m.q);
                        u64* o = Ly.O + ((size_t)(it.ru * Ly.out_groups + gg) * 2 + p) * L * N + (size_t)k * N + x;
                        if (seg > 0) out = addq(out, *o, m.q);  // this thread stored the earlier segments
                        *o = out;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) arrive(ACC_EMPTY);  // accumulators free
            }
            if (!okk) break;
        }
    }
    // drain: after an abort, give in-flight copies and MMAs a bounded time to land before TMEM is freed
    // (after every role has left its loop, so that a wait that gave up late is still reported)
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (*abort_flag && tid == 0) {
        for (u32 i = 0; i < B.n; i++) atomicExch(B.L[i].err, 1);
        for (long long i = 0; i < TC_SPIN_LIMIT / 16; i++) __nanosleep(64);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
    // no CTA leaves while another CTA of its cluster may still copy into its shared memory
    if (CL > 1) asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ------------------------------------------------------------------ operand images, chunk passes
// Step 3, operand-image form with chunk passes, for layers of many output rows.  TMEM holds 512
// columns of fp32 accumulators for the CTA's 128 slots, so five chunk accumulators allow at most
// 102 rows; here a work item takes up to 256 rows and accumulates `cpp` = floor(512 / rows) chunks
// of the residues per pass (two chunks for 256 rows, four for 128, all five for 96 or fewer),
// running ceil(5 / cpp) passes over its K tiles, each copying only its chunks of the images.  A
// 512-row layer then reads each image twice (two 256-row items) instead of six times (six
// 96-row items), and its MMAs have N = 256, the shape that reaches the tensor pipe's peak.  Each
// (pass, segment) accumulation is reduced in the epilogue to sum_c 2^(10 c) (D_c + 512 S) mod q
// over its chunks, put through the Hadamard PMult (linear in A0, A1) and added mod q into the
// output, like the segments of the other forms.  Roles and barriers as in k_mac_img (CL = 1).
constexpr int TCC_STAGES = 4;
constexpr u32 TCC_ROWS = 256;                                   // rows per item at most (MMA N)
constexpr u32 TCC_B_OFF = TCI_A_BYTES;                          // scalar tile after the image chunks
constexpr u32 TCC_STAGE_BYTES = TCI_A_BYTES + TCC_ROWS * TC_KTILE * 2;  // 40 KB + 16 KB
constexpr u32 TCC_BAR_OFF = TCC_STAGES * TCC_STAGE_BYTES;
constexpr u32 TCC_SMEM_BYTES = TCC_BAR_OFF + 128;
static_assert(TCC_SMEM_BYTES <= 227 * 1024, "chunk-pass MAC exceeds shared memory");

__host__ __device__ constexpr u32 tcc_cpp(u32 rows_per_cta) {
    return 512 / rows_per_cta >= (u32)TC_CHUNKS ? (u32)TC_CHUNKS : 512 / rows_per_cta;
}

template <bool PACKED, int MAXB>
__global__ void __launch_bounds__(TC_THREADS, 1) k_mac_cp(const __grid_constant__ Batch<MAXB> B, KP kp) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    constexpr int NR = PACKED ? 2 : 1;
    constexpr int NB = 2 * TCC_STAGES + 2;
    const u32 N = kp.N, L = kp.L, NT = N / TC_MTILE;
    const u32 tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    u64* bars = reinterpret_cast<u64*>(tsm + TCC_BAR_OFF);
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    constexpr int FULL = 0, EMPTY = TCC_STAGES, ACC_FULL = 2 * TCC_STAGES, ACC_EMPTY = 2 * TCC_STAGES + 1;
    u32* tmem_slot = reinterpret_cast<u32*>(tsm + TCC_BAR_OFF + NB * 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tsm + TCC_BAR_OFF + NB * 8 + 4);

    if (tid == 0) {
        for (int i = 0; i < TCC_STAGES; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(FULL + i)), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(EMPTY + i)), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(ACC_FULL)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(ACC_EMPTY)), "r"(TC_EPI));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const u32 tmem = *tmem_slot;

    auto wait = [&](int i, u32 parity) -> bool {
        return mbar_wait_bounded(bar(i), parity, TC_SPIN_LIMIT, abort_flag, nullptr);
    };
    auto arrive = [&](int i) { asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(i)) : "memory"); };

    if (warp == 0) {
        // ---------------------------------------------------------------- copies
        u32 g = 0;
        TcItem it;
        bool ok = true;
        for (u32 item = blockIdx.x; ok && tc_item(B, item, N, L, it); item += gridDim.x) {
            const LayerDev& Ly = *it.ly;
            const u32 rpc = Ly.tc_rows_per_cta, cpp = tcc_cpp(rpc), bbytes = rpc * TC_KTILE * 2;
            const u32 ktiles = Ly.Kpad / TC_KTILE, mt = it.row0 / rpc, nt = it.n0 / TC_MTILE;
            const unsigned char* abase = reinterpret_cast<const unsigned char*>(
                Ly.A16 + ((((size_t)it.ru * 2 + it.p) * L + it.k) * NT + nt) * ktiles * IMG_HALVES);
            for (u32 c0 = 0; ok && c0 < (u32)TC_CHUNKS; c0 += cpp) {
                const u32 ncp = min(cpp, (u32)TC_CHUNKS - c0);
                for (u32 t = 0; t < it.n_tiles; t++, g++) {
                    const u32 s = g % TCC_STAGES;
                    const bool fr = g < TCC_STAGES || wait(EMPTY + s, ((g / TCC_STAGES) - 1) & 1);
                    if (!__all_sync(0xffffffffu, fr)) { ok = false; break; }
                    if (lane == 0) {
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(FULL + s)),
                                     "r"(ncp * TC_A_CHUNK_BYTES + bbytes)
                                     : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                smem_u32(tsm + s * TCC_STAGE_BYTES)),
                            "l"(abase + (size_t)t * TCI_A_BYTES + c0 * TC_A_CHUNK_BYTES), "r"(ncp * TC_A_CHUNK_BYTES),
                            "r"(bar(FULL + s))
                            : "memory");
                        const __half* bsrc = Ly.sc16 + ((size_t)mt * ktiles + t) * (rpc * TC_KTILE);
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                smem_u32(tsm + s * TCC_STAGE_BYTES + TCC_B_OFF)),
                            "l"(bsrc), "r"(bbytes), "r"(bar(FULL + s))
                            : "memory");
                    }
                    __syncwarp();
                }
            }
            if (*abort_flag) ok = false;
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMAs (lane 0)
        if (lane == 0) {
            u32 g = 0, unit = 0;  // unit = (item, pass, segment): one accumulation in TMEM
            TcItem it;
            bool okk = true;
            for (u32 item = blockIdx.x; okk && tc_item(B, item, N, L, it); item += gridDim.x) {
                const u32 idesc = tc_idesc(TC_MTILE, it.nrows), cpp = tcc_cpp(it.ly->tc_rows_per_cta);
                for (u32 c0 = 0; okk && c0 < (u32)TC_CHUNKS; c0 += cpp) {
                    const u32 ncp = min(cpp, (u32)TC_CHUNKS - c0);
                    for (u32 t = 0; t < it.n_tiles; t++, g++) {
                        const u32 s = g % TCC_STAGES, tseg = t % TC_SEG_TILES;
                        if (tseg == 0) {
                            if (unit > 0 && !wait(ACC_EMPTY, (unit - 1) & 1)) { okk = false; break; }
                            asm volatile("tcgen05.fence::after_thread_sync;");
                        }
                        if (!wait(FULL + s, (g / TCC_STAGES) & 1)) { okk = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const u32 a_base = smem_u32(tsm + s * TCC_STAGE_BYTES), b_base = a_base + TCC_B_OFF;
                        for (u32 c = 0; c < ncp; c++) {
#pragma unroll
                            for (int ks = 0; ks < TC_KTILE / 16; ks++) {
                                const u64 ad = smem_desc(a_base + c * TC_A_CHUNK_BYTES + ks * 256);
                                const u64 bd = smem_desc(b_base + ks * 256);
                                const u32 acc = (tseg > 0 || ks > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + c * it.nrows),
                                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                            }
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            bar(EMPTY + s)));
                        if (tseg == TC_SEG_TILES - 1 || t + 1 == it.n_tiles) {
                            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                bar(ACC_FULL)));
                            unit++;
                        }
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ---------------------------------------------------------------- epilogue
        u32 unit = 0;
        TcItem it;
        bool okk = true;
        for (u32 item = blockIdx.x; okk && tc_item(B, item, N, L, it); item += gridDim.x) {
            const LayerDev& Ly = *it.ly;
            const u32 n_seg = (it.n_tiles + TC_SEG_TILES - 1) / TC_SEG_TILES, cpp = tcc_cpp(Ly.tc_rows_per_cta);
            const u32 sp = warp & 3, third = (warp - 4) >> 2;
            const u32 nl = sp * 32 + lane, x = it.n0 + nl, nrows = it.nrows, row0 = it.row0, k = it.k, p = it.p;
            const LimbC m = kp.limb[k];
            const u64 pkv = PACKED ? Ly.pk[(size_t)k * N + x] : 0, pksv = PACKED ? Ly.pksh[(size_t)k * N + x] : 0;
            for (u32 c0 = 0; okk && c0 < (u32)TC_CHUNKS; c0 += cpp) {
                const u32 ncp = min(cpp, (u32)TC_CHUNKS - c0);
                for (u32 seg = 0; seg < n_seg; seg++) {
                    if (!__all_sync(0xffffffffu, wait(ACC_FULL, unit & 1))) { okk = false; break; }
                    unit++;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const bool first = c0 == 0 && seg == 0;
                    for (u32 cb = third * 8; cb < nrows; cb += 24) {
                        u32 d[TC_CHUNKS][8];
#pragma unroll
                        for (int c = 0; c < TC_CHUNKS; c++) {
                            if ((u32)c >= ncp) break;
                            const u32 ta = tmem + ((sp * 32u) << 16) + (u32)c * nrows + cb;
                            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                         : "=r"(d[c][0]), "=r"(d[c][1]), "=r"(d[c][2]), "=r"(d[c][3]), "=r"(d[c][4]),
                                           "=r"(d[c][5]), "=r"(d[c][6]), "=r"(d[c][7])
                                         : "r"(ta));
                        }
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        u64 red[8];
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            const long long b = Ly.bias[(size_t)seg * Ly.tc_rows + row0 + cb + j];  // 512 S of the segment
                            // this pass's chunks of A = hi 2^30 + lo (chunks 0..2 in lo, 3..4 in hi)
                            long long lo = 0, hi = 0;
#pragma unroll
                            for (int c = 0; c < TC_CHUNKS; c++) {
                                if ((u32)c >= ncp) break;
                                const long long v = (long long)__float2int_rn(__uint_as_float(d[c][j])) + b;
                                const u32 e = c0 + c;
                                if (e < 3) lo += v << (10 * e);
                                else hi += v << (10 * (e - 3));
                            }
                            red[j] = tc_reduce(lo, hi, m);
                        }
#pragma unroll
                        for (int j = 0; j < 8; j += NR) {
                            const u32 row = row0 + cb + j;
                            const u32 gg = row / NR;
                            if (gg >= Ly.out_groups) continue;
                            u64 out = red[j];
                            if (PACKED) out = addq(mulmod_shoup(out, kp.kmul, m.ksh, m.q), mulmod_shoup(red[j + 1], pkv, pksv, m.q), m.q);
                            u64* o = Ly.O + ((size_t)(it.ru * Ly.out_groups + gg) * 2 + p) * L * N + (size_t)k * N + x;
                            if (!first) out = addq(out, *o, m.q);  // this thread stored the earlier accumulations
                            *o = out;
                        }
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    __syncwarp();
                    if (lane == 0) arrive(ACC_EMPTY);  // accumulators free
                }
            }
        }
    }
    // drain: after an abort, give in-flight copies and MMAs a bounded time to land before TMEM is freed
    // (after every role has left its loop, so that a wait that gave up late is still reported)
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (*abort_flag && tid == 0) {
        for (u32 i = 0; i < B.n; i++) atomicExch(B.L[i].err, 1);
        for (long long i = 0; i < TC_SPIN_LIMIT / 16; i++) __nanosleep(64);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ------------------------------------------------------------------ operand images, CTA pairs
// Step 3, operand-image form on CTA pairs (tcgen05 cta_group::2), for layers of many output rows.
// The roles of the operands swap: the scalar rows are the MMA's M dimension (128 rows in each
// CTA, 256 per pair) and the NTT slots its N dimension (64 per pair; each CTA holds 32 of them),
// so per K tile a CTA copies an 8 KB scalar tile and 10 KB of image (five chunks of 32 slots)
// for 128 x 64 x 32 products per chunk.  Rows of a CTA's tile are ordered diagonal-major: row
// l < 64 is (group g0 + l, diagonal 0), row 64 + l is (group g0 + l, diagonal 1) (unpacked: row l
// is group g0 + l).  An item is (row unit, polynomial, limb, 64-slot tile, 256-row pair tile).
// Roles: warp 0 copies (both CTAs, tensor copies with .cta_group::2 so that CTA 1's copies complete
// on CTA 0's barrier); warp 1 issues the MMAs (lane 0 of CTA 0); warps 4..15 run the epilogue.
// Barriers (all bounded waits):
//   full[s]    CTA 0 only: both CTAs' copies of stream position g landed in stage s (CTA 0 arrives
//              once and expects the bytes of both)
//   empty[s]   the pair's MMAs of stage s done (commit, multicast to both CTAs)
//   acc_full   last MMA of an accumulation segment done (commit, multicast)
//   acc_empty  CTA 0 only: accumulators of both CTAs read (every epilogue warp of both CTAs)
//   xf[t], xe[t]  packed layers: diagonal-1 products handed to the diagonal-0 warps of column
//                 group t (xf: written, xe: consumed), through a 4 KB exchange buffer per t
constexpr int TCP_STAGES = 10;
constexpr u32 TCP_N = 64;                                   // NTT slots per pair (MMA N)
constexpr u32 TCP_ROWS = 128;                               // scalar rows per CTA (half the MMA M)
constexpr u32 TCP_A_BYTES = TCP_ROWS * TC_KTILE * 2;        // 8 KB scalar tile
constexpr u32 TCP_B_CHUNK = (TCP_N / 2) * TC_KTILE * 2;     // 2 KB: 32 slots x 32 terms of one chunk
constexpr u32 TCP_STAGE_BYTES = TCP_A_BYTES + TC_CHUNKS * TCP_B_CHUNK;  // 18 KB
constexpr u32 TCP_X_OFF = TCP_STAGES * TCP_STAGE_BYTES;
constexpr u32 TCP_X_BYTES = 3 * 64 * 8 * 8;                 // [column group][group][8 slots] u64
constexpr u32 TCP_BAR_OFF = TCP_X_OFF + TCP_X_BYTES;
constexpr int TCP_NB = 2 * TCP_STAGES + 2 + 6;
constexpr u32 TCP_SMEM_BYTES = TCP_BAR_OFF + TCP_NB * 8 + 16;
static_assert(TCP_SMEM_BYTES <= 227 * 1024, "CTA-pair MAC exceeds shared memory");

// item of the CTA-pair MAC: layer, row unit, polynomial, limb, first slot, pair tile
template <int MAXB>
__device__ __forceinline__ bool tcp_item(const Batch<MAXB>& B, u32 item, u32 N, u32 L, TcItem& it) {
    if (item >= B.start[ST_MAC][B.n]) return false;
    const u32 li = find_layer(B, ST_MAC, item);
    const LayerDev& Ly = B.L[li];
    const u32 npairs = (Ly.tc_rows + 2 * TCP_ROWS - 1) / (2 * TCP_ROWS), nn = N / TCP_N;
    const u32 local = item - B.start[ST_MAC][li];
    const u32 pt = local % npairs, n64 = (local / npairs) % nn, z = local / (npairs * nn);
    it.ly = &Ly;
    it.k = z % L, it.p = (z / L) & 1, it.ru = z / (2 * L);
    it.n0 = n64 * TCP_N;
    it.row0 = pt;  // the pair tile
    it.nrows = 2 * TCP_ROWS;
    it.n_tiles = Ly.Kpad / TC_KTILE;
    return true;
}

// bounded wait on a barrier that threads of the other CTA of the pair arrive at
__device__ __forceinline__ bool mbar_wait_cluster(u32 bar, u32 parity, long long limit, volatile int* abort_flag) {
    for (long long it = 0; it < limit; it++) {
        if (*abort_flag) return false;
        u32 ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    *abort_flag = 1;
    return false;
}

// arrive on the barrier at the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ void mbar_arrive_remote(u32 bar, u32 rank) {
    u32 remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(bar), "r"(rank));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

template <bool PACKED, int MAXB>
__global__ void __launch_bounds__(TC_THREADS, 1) k_mac_pair(const __grid_constant__ Batch<MAXB> B, KP kp) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    const u32 N = kp.N, L = kp.L, NT = N / TC_MTILE;
    const u32 tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    u32 rank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const u32 cid = blockIdx.x / 2, n_cl = gridDim.x / 2;
    u64* bars = reinterpret_cast<u64*>(tsm + TCP_BAR_OFF);
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    constexpr int FULL = 0, EMPTY = TCP_STAGES, ACC_FULL = 2 * TCP_STAGES,
                  ACC_EMPTY = ACC_FULL + 1, XF = ACC_FULL + 2, XE = XF + 3;
    u32* tmem_slot = reinterpret_cast<u32*>(tsm + TCP_BAR_OFF + TCP_NB * 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tsm + TCP_BAR_OFF + TCP_NB * 8 + 4);
    u64* xch = reinterpret_cast<u64*>(tsm + TCP_X_OFF);

    if (tid == 0) {
        for (int i = 0; i < TCP_STAGES; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(FULL + i)), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(EMPTY + i)), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(ACC_FULL)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(ACC_EMPTY)), "r"(2 * TC_EPI));
        for (int t = 0; t < 3; t++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(XF + t)), "r"(2));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(XE + t)), "r"(2));
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        // the pair's accumulators: one warp of each CTA allocates, collectively, the same columns in both
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    // both CTAs' barriers are initialised before either copies, commits or arrives across the pair
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;");
    const u32 tmem = *tmem_slot;

    auto wait = [&](int i, u32 parity) -> bool {
        return mbar_wait_bounded(bar(i), parity, TC_SPIN_LIMIT, abort_flag, nullptr);
    };
    auto wait_cl = [&](int i, u32 parity) -> bool { return mbar_wait_cluster(bar(i), parity, TC_SPIN_LIMIT, abort_flag); };

    if (warp == 0) {
        // ---------------------------------------------------------------- copies (both CTAs)
        u32 g = 0;
        TcItem it;
        bool ok = true;
        u32 full0;  // CTA 0's full barriers, as shared::cluster addresses
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(full0) : "r"(bar(FULL)), "r"(0));
        for (u32 item = cid; ok && tcp_item(B, item, N, L, it); item += n_cl) {
            const LayerDev& Ly = *it.ly;
            const u32 ktiles = Ly.Kpad / TC_KTILE, mt = it.row0 * 2 + rank;
            // this CTA's 32 slots of the 64: quarter (n0 mod 128) / 32 + rank of image tile n0 / 128
            const u32 quarter = (it.n0 % TC_MTILE) / (TCP_N / 2) + rank;
            const u32 img0 = (((it.ru * 2 + it.p) * L + it.k) * NT + it.n0 / TC_MTILE) * ktiles;
            for (u32 t = 0; t < it.n_tiles; t++, g++) {
                const u32 s = g % TCP_STAGES;
                const bool fr = g < TCP_STAGES || wait(EMPTY + s, ((g / TCP_STAGES) - 1) & 1);
                if (!__all_sync(0xffffffffu, fr)) { ok = false; break; }
                if (lane == 0) {
                    const u32 st = smem_u32(tsm + s * TCP_STAGE_BYTES), fb = full0 + s * 8;
                    if (rank == 0)
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(FULL + s)),
                                     "r"(2 * TCP_STAGE_BYTES)
                                     : "memory");
                    // scalar tile (mt, t): rows (mt ktiles + t) 16 .. + 15 of 512 bytes
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
                        " [%0], [%1, {%2, %3}], [%4];" ::"r"(st),
                        "l"(&Ly.smap), "r"(0), "r"((mt * ktiles + t) * 16), "r"(fb)
                        : "memory");
                    // image (img0 + t): core-matrix rows 4 quarter .. + 3 of every chunk
                    asm volatile(
                        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
                        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(st + TCP_A_BYTES),
                        "l"(&Ly.rmap), "r"(0), "r"(4 * quarter), "r"(0), "r"(img0 + t), "r"(fb)
                        : "memory");
                }
                __syncwarp();
            }
            if (*abort_flag) ok = false;
        }
        // the other CTA's MMAs commit to this CTA's empty barriers: wait for the commits of the last
        // uses of every stage, so none is still on its way when this CTA leaves
        if (ok) {
            for (u32 gg = g > TCP_STAGES ? g - TCP_STAGES : 0; gg < g; gg++)
                if (!__all_sync(0xffffffffu, wait(EMPTY + gg % TCP_STAGES, (gg / TCP_STAGES) & 1))) break;
        }
    } else if (warp == 1 && rank == 0) {
        // ---------------------------------------------------------------- MMAs (CTA 0, lane 0)
        if (lane == 0) {
            u32 g = 0, unit = 0;
            TcItem it;
            const u32 idesc = tc_idesc(2 * TCP_ROWS, TCP_N);
            for (u32 item = cid; tcp_item(B, item, N, L, it); item += n_cl) {
                bool okk = true;
                for (u32 t = 0; t < it.n_tiles; t++, g++) {
                    const u32 s = g % TCP_STAGES, tseg = t % TC_SEG_TILES;
                    if (tseg == 0) {
                        if (unit > 0 && !wait_cl(ACC_EMPTY, (unit - 1) & 1)) { okk = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                    }
                    if (!wait(FULL + s, (g / TCP_STAGES) & 1)) { okk = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const u32 st = smem_u32(tsm + s * TCP_STAGE_BYTES);
#pragma unroll
                    for (int c = 0; c < TC_CHUNKS; c++) {
#pragma unroll
                        for (int ks = 0; ks < TC_KTILE / 16; ks++) {
                            const u64 ad = smem_desc(st + ks * 256);
                            const u64 bd = smem_desc(st + TCP_A_BYTES + c * TCP_B_CHUNK + ks * 256);
                            const u32 acc = (tseg > 0 || ks > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + c * TCP_N),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                        }
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
                        " [%0], %1;" ::"r"(bar(EMPTY + s)),
                        "h"((uint16_t)3));
                    if (tseg == TC_SEG_TILES - 1 || t + 1 == it.n_tiles) {
                        asm volatile(
                            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
                            " [%0], %1;" ::"r"(bar(ACC_FULL)),
                            "h"((uint16_t)3));
                        unit++;
                    }
                }
                if (!okk) break;
            }
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ---------------------------------------------------------------- epilogue (both CTAs)
        // warp (sp, t): TMEM lanes 32 sp .. + 31 (rows), column groups of 8 slots t, t + 3, t + 6
        const u32 sp = warp & 3, t = (warp - 4) >> 2, rl = sp * 32 + lane;
        const bool diag1 = PACKED && rl >= 64;
        u32 unit = 0, xn = 0;  // accumulation units; exchanges of this column group
        TcItem it;
        for (u32 item = cid; tcp_item(B, item, N, L, it); item += n_cl) {
            const LayerDev& Ly = *it.ly;
            const u32 n_seg = (it.n_tiles + TC_SEG_TILES - 1) / TC_SEG_TILES;
            const u32 gl = PACKED ? (rl & 63) : rl;
            const u32 g = it.row0 * (PACKED ? TCP_ROWS : 2 * TCP_ROWS) + rank * (PACKED ? 64 : TCP_ROWS) + gl;
            const bool live = g < Ly.out_groups;
            const u32 row = PACKED ? g * 2 + (diag1 ? 1 : 0) : g;  // the row in the scalar matrix
            const u32 k = it.k, p = it.p;
            const LimbC m = kp.limb[k];
            bool okk = true;
            for (u32 seg = 0; seg < n_seg && okk; seg++) {
                if (!__all_sync(0xffffffffu, wait(ACC_FULL, unit & 1))) { okk = false; break; }
                unit++;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const long long b = live ? Ly.bias[(size_t)seg * Ly.tc_rows + row] : 0;  // 512 S of the segment
                for (u32 cb = t; cb < TCP_N / 8; cb += 3) {
                    u32 d[TC_CHUNKS][8];
#pragma unroll
                    for (int c = 0; c < TC_CHUNKS; c++) {
                        const u32 ta = tmem + ((sp * 32u) << 16) + (u32)(c * TCP_N) + cb * 8;
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                     : "=r"(d[c][0]), "=r"(d[c][1]), "=r"(d[c][2]), "=r"(d[c][3]), "=r"(d[c][4]),
                                       "=r"(d[c][5]), "=r"(d[c][6]), "=r"(d[c][7])
                                     : "r"(ta));
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    u64 red[8];
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const long long lo = ((long long)__float2int_rn(__uint_as_float(d[0][j])) + b) +
                                             (((long long)__float2int_rn(__uint_as_float(d[1][j])) + b) << 10) +
                                             (((long long)__float2int_rn(__uint_as_float(d[2][j])) + b) << 20);
                        const long long hi = ((long long)__float2int_rn(__uint_as_float(d[3][j])) + b) +
                                             (((long long)__float2int_rn(__uint_as_float(d[4][j])) + b) << 10);
                        const i128 a = (i128)lo + ((i128)hi << 30) + ((i128)m.q << 40);
                        red[j] = bred128((u128)a, m);
                    }
                    const u32 x0 = it.n0 + cb * 8;
                    u64* xb = xch + ((size_t)t * 64 + gl) * 8;
                    if (PACKED && diag1) {
                        // A1 NTT(P_k) to the diagonal-0 thread of the same group and slots
                        if (xn > 0 && !__all_sync(0xffffffffu, wait(XE + t, (xn - 1) & 1))) { okk = false; break; }
#pragma unroll
                        for (int j = 0; j < 8; j++) xb[j] = mulmod(red[j], Ly.pk[(size_t)k * N + x0 + j], m);
                        __syncwarp();
                        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(XF + t)) : "memory");
                        xn++;
                        continue;
                    }
                    u64 add[8];
                    if (PACKED) {
                        if (!__all_sync(0xffffffffu, wait(XF + t, xn & 1))) { okk = false; break; }
#pragma unroll
                        for (int j = 0; j < 8; j++) add[j] = xb[j];
                        __syncwarp();
                        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(XE + t)) : "memory");
                        xn++;
                    }
                    if (live) {
                        u64* o = Ly.O + ((size_t)(it.ru * Ly.out_groups + g) * 2 + p) * L * N + (size_t)k * N + x0;
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            u64 out = PACKED ? addq(mulmod(kp.kmul, red[j], m), add[j], m.q) : red[j];
                            if (seg > 0) out = addq(out, o[j], m.q);  // this thread stored the earlier segments
                            o[j] = out;
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) {
                    if (rank == 0) asm volatile("mbarrier.arrive.release.cluster.shared::cta.b64 _, [%0];" ::"r"(bar(ACC_EMPTY)) : "memory");
                    else mbar_arrive_remote(bar(ACC_EMPTY), 0);
                }
            }
            if (!okk) break;
        }
    }
    // drain: after an abort, give in-flight copies and MMAs a bounded time to land before TMEM is freed
    // (after every role has left its loop, so that a wait that gave up late is still reported)
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (*abort_flag && tid == 0) {
        for (u32 i = 0; i < B.n; i++) atomicExch(B.L[i].err, 1);
        for (long long i = 0; i < TC_SPIN_LIMIT / 16; i++) __nanosleep(64);
    }
    // no CTA frees the pair's accumulators or leaves while the other may still arrive at its barriers
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ------------------------------------------------------------------ fused key switch + MAC
// For layers whose output rows fit one CTA (at most 96 rows, one row tile), the key switch runs
// inside the tensor-core MAC: producer warps compute, per K tile, the 32 rotated residues of the
// tile's 128 destination slots and write their fp16 chunks straight into the shared-memory
// operand stage the MMA reads, so rotated copies never leave the SM (Sec. 3.1: the hoisted
// rotations feed the CMult/HAdd sum directly; Sec. 3.2.2: one reduction per lazy sum).
// Roles: warp 0 copies the scalar tiles, warp 1 (lane 0) issues the MMAs, warps 2..17 produce
// operands (four groups of 128 threads, eight consecutive terms each per K tile; a thread owns
// a SOURCE slot, as in k_keyswitch) and run the epilogue.  Barriers (all bounded waits):
//   full[s]    producers wrote stage s (16 warp arrivals) and its scalar tile landed (1 + tx)
//   empty[s]   MMAs of stage s done (commit)
//   acc_full / acc_empty as in k_mac_img.
constexpr int KF_PROD_WARPS = 16;
constexpr int KF_THREADS = (2 + KF_PROD_WARPS) * 32;
constexpr int KF_STAGES = 3;
constexpr u32 KF_B_OFF = KF_STAGES * TCI_A_BYTES;
constexpr u32 KF_BAR_OFF = KF_B_OFF + KF_STAGES * TC_B_BYTES;
constexpr u32 KF_SMEM_BYTES = KF_BAR_OFF + 128;
static_assert(KF_SMEM_BYTES <= 227 * 1024, "fused MAC exceeds shared memory");

template <bool PACKED, int LL, int MAXB>
__global__ void __launch_bounds__(KF_THREADS, 1) k_ksmac(const __grid_constant__ Batch<MAXB> B, KP kp, u32 tmem_cols) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    constexpr int NR = PACKED ? 2 : 1;
    constexpr int NB = 2 * KF_STAGES + 2;
    constexpr int FULL = 0, EMPTY = KF_STAGES, ACC_FULL = 2 * KF_STAGES, ACC_EMPTY = 2 * KF_STAGES + 1;
    const u32 N = kp.N, L = kp.L, logN = kp.logN;
    const u32 tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    u64* bars = reinterpret_cast<u64*>(tsm + KF_BAR_OFF);
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    u32* tmem_slot = reinterpret_cast<u32*>(tsm + KF_BAR_OFF + NB * 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tsm + KF_BAR_OFF + NB * 8 + 4);

    if (tid == 0) {
        for (int i = 0; i < KF_STAGES; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(FULL + i)), "r"(KF_PROD_WARPS + 1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(EMPTY + i)), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(ACC_FULL)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(ACC_EMPTY)), "r"(KF_PROD_WARPS));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const u32 tmem = *tmem_slot;
    auto wait = [&](int i, u32 parity) -> bool {
        return mbar_wait_bounded(bar(i), parity, TC_SPIN_LIMIT, abort_flag, nullptr);
    };
    auto arrive = [&](int i) { asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(i)) : "memory"); };

    if (warp == 0) {
        // ---------------------------------------------------------------- scalar tiles
        u32 g = 0;
        TcItem it;
        bool ok = true;
        for (u32 item = blockIdx.x; ok && tc_item(B, item, N, L, it); item += gridDim.x) {
            const LayerDev& Ly = *it.ly;
            const u32 bbytes = Ly.tc_rows_per_cta * TC_KTILE * 2, ktiles = Ly.Kpad / TC_KTILE;
            for (u32 t = 0; t < it.n_tiles; t++, g++) {
                const u32 s = g % KF_STAGES;
                const bool fr = g < KF_STAGES || wait(EMPTY + s, ((g / KF_STAGES) - 1) & 1);
                if (!__all_sync(0xffffffffu, fr)) { ok = false; break; }
                if (lane == 0) {
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(FULL + s)), "r"(bbytes)
                                 : "memory");
                    const __half* bsrc = Ly.sc16 + (size_t)t * (Ly.tc_rows_per_cta * TC_KTILE);
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(tsm + KF_B_OFF + s * TC_B_BYTES)),
                        "l"(bsrc), "r"(bbytes), "r"(bar(FULL + s))
                        : "memory");
                }
                __syncwarp();
            }
            (void)ktiles;
            if (*abort_flag) ok = false;
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMAs (lane 0)
        if (lane == 0) {
            u32 g = 0, unit = 0;
            TcItem it;
            for (u32 item = blockIdx.x; tc_item(B, item, N, L, it); item += gridDim.x) {
                const u32 idesc = tc_idesc(TC_MTILE, it.nrows);
                bool okk = true;
                for (u32 t = 0; t < it.n_tiles; t++, g++) {
                    const u32 s = g % KF_STAGES, tseg = t % TC_SEG_TILES;
                    if (tseg == 0) {
                        if (unit > 0 && !wait(ACC_EMPTY, (unit - 1) & 1)) { okk = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                    }
                    if (!wait(FULL + s, (g / KF_STAGES) & 1)) { okk = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const u32 a_base = smem_u32(tsm + s * TCI_A_BYTES), b_base = smem_u32(tsm + KF_B_OFF + s * TC_B_BYTES);
#pragma unroll
                    for (int c = 0; c < TC_CHUNKS; c++) {
#pragma unroll
                        for (int ks = 0; ks < TC_KTILE / 16; ks++) {
                            const u64 ad = smem_desc(a_base + c * TC_A_CHUNK_BYTES + ks * 256);
                            const u64 bd = smem_desc(b_base + ks * 256);
                            const u32 acc = (tseg > 0 || ks > 0) ? 1u : 0u;
                            const u32 dt = tmem + (u32)(c * it.nrows);
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        bar(EMPTY + s)));
                    if (tseg == TC_SEG_TILES - 1 || t + 1 == it.n_tiles) {
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            bar(ACC_FULL)));
                        unit++;
                    }
                }
                if (!okk) break;
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- producers + epilogue
        const u32 pt = tid - 64, grp = pt >> 7, t = pt & (TC_MTILE - 1);  // group of 8 terms, slot in tile
        u32 g = 0, unit = 0;
        TcItem it;
        for (u32 item = blockIdx.x; tc_item(B, item, N, L, it); item += gridDim.x) {
            const LayerDev& Ly = *it.ly;
            const u32 k = it.k, p = it.p, nt = it.n0 / TC_MTILE;
            const LimbC m = kp.limb[k];
            const int red = m.sm1 == 49 ? (m.delta ? 1 : 2) : 3;
            const size_t ctw = 2ull * L * N, d_step = (size_t)LL * L * N, dd_step = (size_t)L * N;
            const size_t r_step = (size_t)Ly.r_slots * ctw;
            const u32 nterm = Ly.n_rot_all * Ly.in_pad;
            u32 cur_rot = ~0u, y = 0, xl = t, src_base = 0;
            u32 kl_[LL], kh_[LL];
            bool ident = false;
            bool okk = true;
            for (u32 tt = 0; tt < it.n_tiles; tt++, g++) {
                const u32 s = g % KF_STAGES;
                const bool fr = g < KF_STAGES || wait(EMPTY + s, ((g / KF_STAGES) - 1) & 1);
                if (!__all_sync(0xffffffffu, fr)) { okk = false; break; }
                unsigned char* A = tsm + s * TCI_A_BYTES;
                const u32 kk0 = tt * TC_KTILE + grp * 8;
                u64 v[8];
                u32 row = t;  // the zero terms past the last rotation go to row t
                if (kk0 < nterm) {
                    const u32 r = kk0 / Ly.in_pad, j0 = kk0 % Ly.in_pad;
                    if (r != cur_rot) {
                        // the rotation's source tile for destination tile nt, this thread's source
                        // slot there and its destination x = src^-1(y); the keys of (x, p, limb)
                        const RotDev rd = Ly.rots_all[r];
                        const u32 x0 = nt * TC_MTILE;
                        const u32 e0 = 2 * (__brev(x0) >> (32 - logN)) + 1;
                        const u32 s0 = __brev((u32)((((u64)e0 * rd.galois) & (2ull * N - 1)) - 1) >> 1) >> (32 - logN);
                        src_base = s0 & ~(TC_MTILE - 1);
                        y = src_base + t;
                        const u32 e = 2 * (__brev(y) >> (32 - logN)) + 1;
                        const u32 x = __brev((u32)((((u64)e * rd.galois_inv) & (2ull * N - 1)) - 1) >> 1) >> (32 - logN);
                        xl = x & (TC_MTILE - 1);
                        ident = r == Ly.id_rot;
                        if (!ident) {
                            const u64* kb = Ly.ksk + (size_t)rd.key * LL * 2 * L * N + ((size_t)p * L + k) * N + x;
#pragma unroll
                            for (int dd = 0; dd < LL; dd++) {
                                const u64 a = __ldg(kb + (size_t)dd * 2 * L * N);
                                kl_[dd] = (u32)(a & 0x1FFFFFFu), kh_[dd] = (u32)(a >> 25);
                            }
                        }
                        cur_rot = r;
                    }
                    row = xl;
                    const u32 c_first = it.ru * Ly.in_groups + j0;
                    const u32 nj = j0 >= Ly.in_groups ? 0u : min(8u, Ly.in_groups - j0);
                    const u64* Rp = Ly.R + ((size_t)c_first * Ly.r_slots + Ly.r_id) * ctw + (size_t)k * N + y;
                    const u64* Dp = Ly.D + (size_t)c_first * d_step + (size_t)k * N + y;
                    if (ident) {
#pragma unroll
                        for (int jj = 0; jj < 8; jj++) v[jj] = jj < (int)nj ? __ldg(Rp + jj * r_step + p * dd_step) : 0;
                    } else if (red <= 2) {
#pragma unroll
                        for (int jj = 0; jj < 8; jj++) {
                            v[jj] = 0;
                            if (jj >= (int)nj) continue;
                            const u64* Dc = Dp + jj * d_step;
                            u64 lo = 0, mid = 0, hi = 0;
#pragma unroll
                            for (int dd = 0; dd < LL; dd++) {
                                const u64 dv = __ldg(Dc + dd * dd_step);
                                const u32 dl = (u32)dv, dh = (u32)(dv >> 32);  // stored split at bit 25
                                mad_wide_u(lo, dl, kl_[dd]);
                                mad_wide_u(hi, dh, kh_[dd]);
                                mad_wide_u(mid, dl + dh, kl_[dd] + kh_[dd]);
                            }
                            mid -= lo + hi;
                            if (p == 0) lo += __ldg(Rp + jj * r_step);  // + sigma(c0)
                            v[jj] = red == 1 ? fold_reduce50(lo, mid, hi, m) : bred_split50(lo, mid, hi, m);
                        }
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 8; jj++) {
                            v[jj] = 0;
                            if (jj >= (int)nj) continue;
                            const u64* Dc = Dp + jj * d_step;
                            u64 lo = 0, mid = 0, hi = 0;
#pragma unroll
                            for (int dd = 0; dd < LL; dd++) {
                                const u64 dv = __ldg(Dc + dd * dd_step);
                                const u32 dl = (u32)dv, dh = (u32)(dv >> 32);  // stored split at bit 25
                                mad_wide_u(lo, dl, kl_[dd]);
                                mad_wide_u(mid, dl, kh_[dd]);
                                mad_wide_u(mid, dh, kl_[dd]);
                                mad_wide_u(hi, dh, kh_[dd]);
                            }
                            if (p == 0) lo += __ldg(Rp + jj * r_step);
                            v[jj] = bred128(((u128)hi << 50) + ((u128)mid << 25) + lo, m);
                        }
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < 8; jj++) v[jj] = 0;
                }
                // the eight terms' chunks: row `row`, terms grp*8 .. grp*8+7 of the stage (16 bytes a chunk)
                const u32 off = (row >> 3) * 512 + grp * 128 + (row & 7) * 16;
#pragma unroll
                for (int c = 0; c < TC_CHUNKS; c++) {
                    u64 v4[KSI_JH];
#pragma unroll
                    for (int e = 0; e < KSI_JH; e++) v4[e] = v[e];
                    const uint2 a = chunk_pack4(v4, c);
#pragma unroll
                    for (int e = 0; e < KSI_JH; e++) v4[e] = v[KSI_JH + e];
                    const uint2 b = chunk_pack4(v4, c);
                    *reinterpret_cast<uint4*>(A + c * TC_A_CHUNK_BYTES + off) = make_uint4(a.x, a.y, b.x, b.y);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) arrive(FULL + s);
                if (tt % TC_SEG_TILES != TC_SEG_TILES - 1 && tt + 1 != it.n_tiles) continue;
                // epilogue of segment seg (as k_mac_img; the 16 warps take every fourth 8-row block)
                const u32 seg = tt / TC_SEG_TILES;
                if (!__all_sync(0xffffffffu, wait(ACC_FULL, unit & 1))) { okk = false; break; }
                unit++;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const u32 sp = warp & 3, quarter = (warp - 2) >> 2;
                const u32 nl = sp * 32 + lane, x = it.n0 + nl, nrows = it.nrows, row0 = it.row0;
                const u64 pkv = PACKED ? Ly.pk[(size_t)k * N + x] : 0;
                for (u32 cb = quarter * 8; cb < nrows; cb += 32) {
                    u32 d[TC_CHUNKS][8];
#pragma unroll
                    for (int c = 0; c < TC_CHUNKS; c++) {
                        const u32 ta = tmem + ((sp * 32u) << 16) + (u32)(c * nrows) + cb;
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                     : "=r"(d[c][0]), "=r"(d[c][1]), "=r"(d[c][2]), "=r"(d[c][3]), "=r"(d[c][4]),
                                       "=r"(d[c][5]), "=r"(d[c][6]), "=r"(d[c][7])
                                     : "r"(ta));
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    u64 rr[8];
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const long long b = Ly.bias[(size_t)seg * Ly.tc_rows + row0 + cb + j];
                        const long long lo = ((long long)__float2int_rn(__uint_as_float(d[0][j])) + b) +
                                             (((long long)__float2int_rn(__uint_as_float(d[1][j])) + b) << 10) +
                                             (((long long)__float2int_rn(__uint_as_float(d[2][j])) + b) << 20);
                        const long long hi = ((long long)__float2int_rn(__uint_as_float(d[3][j])) + b) +
                                             (((long long)__float2int_rn(__uint_as_float(d[4][j])) + b) << 10);
                        const i128 a = (i128)lo + ((i128)hi << 30) + ((i128)m.q << 40);
                        rr[j] = bred128((u128)a, m);
                    }
#pragma unroll
                    for (int j = 0; j < 8; j += NR) {
                        const u32 rw = row0 + cb + j;
                        const u32 gg = rw / NR;
                        if (gg >= Ly.out_groups) continue;
                        u64 out = rr[j];
                        if (PACKED) out = addq(mulmod(kp.kmul, out, m), mulmod(rr[j + 1], pkv, m), m.q);
                        u64* o = Ly.O + ((size_t)(it.ru * Ly.out_groups + gg) * 2 + p) * L * N + (size_t)k * N + x;
                        if (seg > 0) out = addq(out, *o, m.q);
                        *o = out;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) arrive(ACC_EMPTY);
            }
            if (!okk) break;
        }
    }
    // (after every role has left its loop, so that a wait that gave up late is still reported)
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (*abort_flag && tid == 0) {
        for (u32 i = 0; i < B.n; i++) atomicExch(B.L[i].err, 1);
        for (long long i = 0; i < TC_SPIN_LIMIT / 16; i++) __nanosleep(64);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
}

// ------------------------------------------------------------------ profiling
struct Prof {
    std::mutex mu;
    bool on = false;
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        CUDA_OK(cudaEventCreate(&e));
        return e;
    }
} g_prof;

struct StageTimer {
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    bool on;
    StageTimer(int st, cudaStream_t str, bool allowed = true) : stage(st), s(str) {
        std::lock_guard<std::mutex> lk(g_prof.mu);
        on = g_prof.on && allowed;
        if (on) {
            a = g_prof.get();
            b = g_prof.get();
            cudaEventRecord(a, s);
        }
    }
    ~StageTimer() {
        if (!on) return;
        cudaEventRecord(b, s);
        std::lock_guard<std::mutex> lk(g_prof.mu);
        g_prof.recs.push_back({stage, a, b});
    }
};

// NVTX range for profilers' timelines (plan, forward, batch); free when no tool is attached
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

void check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(HE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------------ tables
KP make_kp(const he_params* p) {
    const DeviceTables& T = device_tables(p);
    KP kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.N = p->N, kp.logN = p->logN, kp.L = p->L, kp.l = p->l, kp.w = p->w;
    kp.kmul = p->k;
    kp.kmul4 = p->k4;
    for (u32 k = 0; k < p->L; k++) {
        kp.limb[k].q = p->q[k];
        kp.limb[k].mu = p->mod[k].mu;
        kp.limb[k].sm1 = p->mod[k].sm1;
        const u64 d50 = (1ull << 50) - p->q[k];
        kp.limb[k].delta = (p->q[k] < (1ull << 50) && d50 < (1ull << 22)) ? (u32)d50 : 0u;
        kp.limb[k].ninv = p->ntt[k].ninv;
        kp.limb[k].ninv_sh = p->ntt[k].ninv_sh;
        kp.limb[k].ksh = (u64)((((unsigned __int128)(p->k % p->q[k])) << 64) / p->q[k]);
    }
    kp.tw = T.tw, kp.itw = T.itw;
    return kp;
}

u32 ntt_threads(u32 N) { return std::min<u32>(NTT_MAX_THREADS, N / NTT_E); }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
void encode_tiled(CUtensorMap* map, CUtensorMapDataType type, u32 rank, const void* base, const cuuint64_t* dims,
                  const cuuint64_t* strides, const cuuint32_t* box) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    });
    if (!fn) fail(HE_ECUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(map, type, rank, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(HE_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

void encode_rmap(CUtensorMap* map, const u64* R, u32 N, u32 L, u32 rows) {
    const cuuint64_t dims[3] = {N, 2ull * L, rows};
    const cuuint64_t strides[2] = {(cuuint64_t)N * 8, 2ull * L * N * 8};
    const cuuint32_t box[3] = {TC_MTILE, 1, TC_KTILE};
    encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, R, dims, strides, box);
}

// The CTA-pair MAC's copies.  Images as (512-byte core-matrix row of 256 halves, row 0..15 of a
// chunk, chunk 0..4, image), one copy taking 4 rows of each chunk (a CTA's 32 slots, 10 KB);
// scalar tiles as rows of 512 bytes, one copy taking the 16 rows of a tile (8 KB).
void tcp_encode_maps(CUtensorMap* imap, CUtensorMap* smap, const __half* A16, u64 n_img, const __half* sc16,
                     u64 n_tiles) {
    const cuuint64_t idims[4] = {256, 16, TC_CHUNKS, n_img};
    const cuuint64_t istr[3] = {TC_SBO, TC_A_CHUNK_BYTES, TCI_A_BYTES};
    const cuuint32_t ibox[4] = {256, 4, TC_CHUNKS, 1};
    encode_tiled(imap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, A16, idims, istr, ibox);
    const cuuint64_t sdims[2] = {256, n_tiles * 16};
    const cuuint64_t sstr[1] = {512};
    const cuuint32_t sbox[2] = {256, 16};
    encode_tiled(smap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, sc16, sdims, sstr, sbox);
}

int sm_count() {
    int dev = 0, n = 0;
    CUDA_OK(cudaGetDevice(&dev));
    CUDA_OK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    return std::max(n, 1);
}

template <class K>
void allow_smem(K kernel, size_t bytes) {
    CUDA_OK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

void launch_ntt_plain(const he_params* p, const KP& kp, u64* d, int n, int inverse, cudaStream_t s) {
    if (n <= 0) return;
    size_t smem = ntt_smem_bytes(p->N);
    allow_smem(k_ntt_plain, smem);
    k_ntt_plain<<<n, ntt_threads(p->N), smem, s>>>(d, kp, inverse);
    check_launch("k_ntt_plain");
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Uploads Galois keys (coefficient form) and converts them to NTT form.
u64* upload_keys(const he_params* p, const KP& kp, const std::vector<const std::vector<u64>*>& keys,
                 cudaStream_t s) {
    const size_t per = (size_t)p->L * p->l * 2 * p->L * p->N;
    u64* d = nullptr;
    if (keys.empty()) return nullptr;
    CUDA_OK(cudaMalloc(&d, per * keys.size() * 8));
    for (size_t i = 0; i < keys.size(); i++)
        CUDA_OK(cudaMemcpyAsync(d + i * per, keys[i]->data(), per * 8, cudaMemcpyHostToDevice, s));
    launch_ntt_plain(p, kp, d, (int)(keys.size() * per / p->N), 0, s);
    return d;
}

// Residues for timing runs: word i of polynomial j (limb j % L) = SplitMix64(seed + i + j N) mod q.
__global__ void k_fill_uniform(u64* __restrict__ a, size_t n_polys, KP kp, u64 seed) {
    const size_t total = n_polys * kp.N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        u64 z = seed + i * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        a[i] = z % kp.limb[(i / kp.N) % kp.L].q;
    }
}

void fill_uniform(const KP& kp, u64* d, size_t n_polys, u64 seed, cudaStream_t s) {
    if (!n_polys) return;
    k_fill_uniform<<<(u32)std::min<size_t>(4096, (n_polys * kp.N + 255) / 256), 256, 0, s>>>(d, n_polys, kp, seed);
    check_launch("k_fill_uniform");
}

// MAC kernel variants: tensor core (packed or not) or CUDA cores (group tile, packed, depthwise)
struct MacVariant {
    bool tc = false, packed = false, dw = false, eager = false, img = false, fused = false, pair = false, cp = false;
    bool h4 = false;     // c_n = 4: four rows per output group (CUDA-core MAC)
    u32 gt = 8, cl = 1;  // cl: CTAs per cluster of the operand-image MAC
    bool operator==(const MacVariant& o) const {
        return tc == o.tc && packed == o.packed && h4 == o.h4 && dw == o.dw && eager == o.eager && img == o.img && cl == o.cl &&
               fused == o.fused && pair == o.pair && cp == o.cp && (tc || eager || gt == o.gt);
    }
};

struct StageLayer {
    LayerDev dev;
    MacVariant mv;
};

u32 stage_blocks(const he_params* p, const StageLayer& s, int stage) {
    const LayerDev& d = s.dev;
    const u32 L = p->L, N = p->N;
    switch (stage) {
        case ST_NTT: return d.n_ct_in * (L + (p->l == 1 ? 0 : L) + L * p->l * L);
        case ST_KS:
            if (d.img) return d.row_units * ((d.in_pad + KSI_JB - 1) / KSI_JB) * d.ks_rg * L * (N / TC_MTILE);
            return d.n_ks * L * (N / KS_THREADS);
        case ST_MAC:
            if (s.mv.eager) return d.row_units * 2 * L * (N / MAC_THREADS) * ((d.out_groups + 3) / 4);
            if (s.mv.pair) return d.row_units * 2 * L * (N / TCP_N) * ((d.tc_rows + 2 * TCP_ROWS - 1) / (2 * TCP_ROWS));
            if (s.mv.tc)
                return d.row_units * 2 * L * (N / TC_MTILE) * ((d.tc_rows + d.tc_rows_per_cta - 1) / d.tc_rows_per_cta) /
                       s.mv.cl;
            return d.row_units * 2 * L * (N / MAC_THREADS) * ((d.out_groups + s.mv.gt - 1) / s.mv.gt);
        default: return d.n_ct_out * 2 * L;
    }
}

template <int LL, int MAXB>
void ks_launch(u32 blocks, const Batch<MAXB>& B, const KP& kp, cudaStream_t s, bool img) {
    if (img) {
        allow_smem(k_keyswitch_img<LL, MAXB>, ksi_smem_bytes(LL));
        k_keyswitch_img<LL, MAXB><<<blocks, KSI_THREADS, ksi_smem_bytes(LL), s>>>(B, kp);
    }
    else k_keyswitch<LL, MAXB><<<blocks, KS_THREADS, 0, s>>>(B, kp);
}

template <int MAXB>
void launch_keyswitch_b(const he_params* p, u32 blocks, const Batch<MAXB>& B, const KP& kp, cudaStream_t s,
                        bool img) {
    switch (p->L * p->l) {
#define KS_CASE(v) \
    case v: ks_launch<v, MAXB>(blocks, B, kp, s, img); break;
        KS_CASE(1) KS_CASE(2) KS_CASE(3) KS_CASE(4) KS_CASE(5) KS_CASE(6) KS_CASE(7) KS_CASE(8) KS_CASE(9)
            KS_CASE(10) KS_CASE(12) KS_CASE(14) KS_CASE(15) KS_CASE(16)
#undef KS_CASE
        default:
            fail(HE_EINVAL, "L * l must be at most 16 (and not 11 or 13)");
    }
}

template <int GT, int NR, bool DW, int MAXB>
void mac_cuda_launch(u32 blocks, const Batch<MAXB>& B, const KP& kp, cudaStream_t s) {
    k_mac<GT, NR, DW, MAXB><<<blocks, MAC_THREADS, 0, s>>>(B, kp);
}

// Persistent launch of the operand-image MAC in clusters of CL CTAs: as many clusters as fit the
// device at once (one CTA per SM), at most one per cluster item.
template <int CL, int MAXB>
void mac_img_launch(bool packed, u32 items, const Batch<MAXB>& B, const KP& kp, u32 cols, cudaStream_t s) {
    auto kern = packed ? k_mac_img<true, CL, MAXB> : k_mac_img<false, CL, MAXB>;
    allow_smem(kern, TCI_SMEM_BYTES);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = TCI_SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int cached[9] = {0};  // clusters that fit at once, per cluster size (one device per process)
    if (!cached[CL]) {
        int n = 0;
        cfg.gridDim = dim3(CL * 64);
        if (CL == 1 || cudaOccupancyMaxActiveClusters(&n, (void*)kern, &cfg) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = sm_count() / CL;
        }
        cached[CL] = std::max(n, 1);
    }
    const u32 n_cl = std::min<u32>(items, (u32)cached[CL]);
    cfg.gridDim = dim3(n_cl * CL);
    CUDA_OK(cudaLaunchKernelEx(&cfg, kern, B, kp, cols));
}

// Persistent launch of the CTA-pair MAC: as many pairs as fit the device at once, at most one per item.
template <int MAXB>
void mac_pair_launch(bool packed, u32 items, const Batch<MAXB>& B, const KP& kp, cudaStream_t s) {
    auto kern = packed ? k_mac_pair<true, MAXB> : k_mac_pair<false, MAXB>;
    allow_smem(kern, TCP_SMEM_BYTES);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = TCP_SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int cached = 0;  // pairs that fit at once (one device per process)
    if (!cached) {
        int n = 0;
        cfg.gridDim = dim3(128);
        if (cudaOccupancyMaxActiveClusters(&n, (void*)kern, &cfg) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = sm_count() / 2;
        }
        cached = std::max(n, 1);
    }
    cfg.gridDim = dim3(2 * std::min<u32>(items, (u32)cached));
    CUDA_OK(cudaLaunchKernelEx(&cfg, kern, B, kp));
}

template <int LL, int MAXB>
void ksmac_launch(bool packed, u32 grid, const Batch<MAXB>& B, const KP& kp, u32 cols, cudaStream_t s) {
    if (packed) {
        allow_smem(k_ksmac<true, LL, MAXB>, KF_SMEM_BYTES);
        k_ksmac<true, LL, MAXB><<<grid, KF_THREADS, KF_SMEM_BYTES, s>>>(B, kp, cols);
    } else {
        allow_smem(k_ksmac<false, LL, MAXB>, KF_SMEM_BYTES);
        k_ksmac<false, LL, MAXB><<<grid, KF_THREADS, KF_SMEM_BYTES, s>>>(B, kp, cols);
    }
}

template <int MAXB>
void launch_ksmac_b(const he_params* p, bool packed, u32 grid, const Batch<MAXB>& B, const KP& kp, u32 cols,
                    cudaStream_t s) {
    switch (p->L * p->l) {
#define KF_CASE(v) \
    case v: ksmac_launch<v, MAXB>(packed, grid, B, kp, cols, s); break;
        KF_CASE(1) KF_CASE(2) KF_CASE(3) KF_CASE(4) KF_CASE(5) KF_CASE(6) KF_CASE(7) KF_CASE(8) KF_CASE(9)
            KF_CASE(10) KF_CASE(12) KF_CASE(14) KF_CASE(15) KF_CASE(16)
#undef KF_CASE
        default:
            fail(HE_EINVAL, "L * l must be at most 16 (and not 11 or 13)");
    }
}

template <int MAXB>
void launch_mac_b(const he_params* p, const MacVariant& mv, u32 blocks, const Batch<MAXB>& B, const KP& kp,
                  cudaStream_t s) {
    if (mv.eager) {
        if (mv.packed) k_mac_eager<true, MAXB><<<blocks, MAC_THREADS, 0, s>>>(B, kp);
        else k_mac_eager<false, MAXB><<<blocks, MAC_THREADS, 0, s>>>(B, kp);
        return;
    }
    if (mv.tc) {
        // persistent: one CTA per SM (the shared-memory footprint allows one), TMEM for the widest layer
        u32 cols = 32;
        for (u32 i = 0; i < B.n; i++) cols = std::max(cols, B.L[i].tmem_cols);
        const u32 grid = std::min(blocks, (u32)sm_count());
        if (mv.fused) {
            launch_ksmac_b<MAXB>(p, mv.packed, grid, B, kp, cols, s);
            return;
        }
        if (mv.pair) {
            mac_pair_launch<MAXB>(mv.packed, blocks, B, kp, s);
            return;
        }
        if (mv.cp) {
            if (mv.packed) {
                allow_smem(k_mac_cp<true, MAXB>, TCC_SMEM_BYTES);
                k_mac_cp<true, MAXB><<<grid, TC_THREADS, TCC_SMEM_BYTES, s>>>(B, kp);
            } else {
                allow_smem(k_mac_cp<false, MAXB>, TCC_SMEM_BYTES);
                k_mac_cp<false, MAXB><<<grid, TC_THREADS, TCC_SMEM_BYTES, s>>>(B, kp);
            }
            return;
        }
        if (mv.img) {
            switch (mv.cl) {
                case 1: mac_img_launch<1, MAXB>(mv.packed, blocks, B, kp, cols, s); break;
                case 2: mac_img_launch<2, MAXB>(mv.packed, blocks, B, kp, cols, s); break;
                case 4: mac_img_launch<4, MAXB>(mv.packed, blocks, B, kp, cols, s); break;
                default: mac_img_launch<8, MAXB>(mv.packed, blocks, B, kp, cols, s); break;
            }
            return;
        }
        if (mv.packed) {
            allow_smem(k_mac_tc<true, MAXB>, TC_SMEM_BYTES);
            k_mac_tc<true, MAXB><<<grid, TC_THREADS, TC_SMEM_BYTES, s>>>(B, kp, cols);
        } else {
            allow_smem(k_mac_tc<false, MAXB>, TC_SMEM_BYTES);
            k_mac_tc<false, MAXB><<<grid, TC_THREADS, TC_SMEM_BYTES, s>>>(B, kp, cols);
        }
        return;
    }
    if (mv.dw) {
        if (mv.h4) mac_cuda_launch<1, 4, true, MAXB>(blocks, B, kp, s);
        else if (mv.packed) mac_cuda_launch<1, 2, true, MAXB>(blocks, B, kp, s);
        else mac_cuda_launch<1, 1, true, MAXB>(blocks, B, kp, s);
        return;
    }
    if (mv.h4) {
        // four rows per group: at most 4 groups per block (16 accumulator pairs, as 8 pair groups)
        switch (mv.gt) {
            case 1: mac_cuda_launch<1, 4, false, MAXB>(blocks, B, kp, s); break;
            case 2: mac_cuda_launch<2, 4, false, MAXB>(blocks, B, kp, s); break;
            default: mac_cuda_launch<4, 4, false, MAXB>(blocks, B, kp, s); break;
        }
    } else if (mv.packed) {
        switch (mv.gt) {
            case 1: mac_cuda_launch<1, 2, false, MAXB>(blocks, B, kp, s); break;
            case 2: mac_cuda_launch<2, 2, false, MAXB>(blocks, B, kp, s); break;
            case 4: mac_cuda_launch<4, 2, false, MAXB>(blocks, B, kp, s); break;
            default: mac_cuda_launch<8, 2, false, MAXB>(blocks, B, kp, s); break;
        }
    } else {
        switch (mv.gt) {
            case 1: mac_cuda_launch<1, 1, false, MAXB>(blocks, B, kp, s); break;
            case 2: mac_cuda_launch<2, 1, false, MAXB>(blocks, B, kp, s); break;
            case 4: mac_cuda_launch<4, 1, false, MAXB>(blocks, B, kp, s); break;
            case 8: mac_cuda_launch<8, 1, false, MAXB>(blocks, B, kp, s); break;
            default: mac_cuda_launch<16, 1, false, MAXB>(blocks, B, kp, s); break;
        }
    }
}

// Launches one stage over the given layers in tables of at most MAXB layers.
template <int MAXB>
void launch_stage(const he_params* p, const KP& kp, int stage, const std::vector<const StageLayer*>& layers,
                  cudaStream_t s) {
    for (size_t c0 = 0; c0 < layers.size(); c0 += MAXB) {
        const u32 n = (u32)std::min<size_t>(MAXB, layers.size() - c0);
        Batch<MAXB> B;
        std::memset(&B, 0, sizeof(B));
        B.n = n;
        u32 total = 0;
        for (u32 i = 0; i < n; i++) {
            B.L[i] = layers[c0 + i]->dev;
            B.start[stage][i] = total;
            total += stage_blocks(p, *layers[c0 + i], stage);
        }
        B.start[stage][n] = total;
        if (!total) continue;
        switch (stage) {
            case ST_NTT: {
                const size_t smem = ntt_smem_bytes(p->N);
                if (p->N >= NTT_BIG_N) {
                    allow_smem(k_ntt_inputs<MAXB, NTT_BIG_THREADS, 1>, smem);
                    k_ntt_inputs<MAXB, NTT_BIG_THREADS, 1><<<total, NTT_BIG_THREADS, smem, s>>>(B, kp);
                } else {
                    allow_smem(k_ntt_inputs<MAXB, NTT_MAX_THREADS, 2>, smem);
                    k_ntt_inputs<MAXB, NTT_MAX_THREADS, 2><<<total, ntt_threads(p->N), smem, s>>>(B, kp);
                }
                check_launch("k_ntt_inputs");
                break;
            }
            case ST_KS:
                launch_keyswitch_b<MAXB>(p, total, B, kp, s, layers[c0]->dev.img != 0);
                check_launch("k_keyswitch");
                break;
            case ST_MAC:
                launch_mac_b<MAXB>(p, layers[c0]->mv, total, B, kp, s);
                check_launch("k_mac");
                break;
            default: {
                const size_t smem = ntt_smem_bytes(p->N);
                if (p->N >= NTT_BIG_N) {
                    allow_smem(k_intt<MAXB, NTT_BIG_THREADS, 1>, smem);
                    k_intt<MAXB, NTT_BIG_THREADS, 1><<<total, NTT_BIG_THREADS, smem, s>>>(B, kp);
                } else {
                    allow_smem(k_intt<MAXB, NTT_MAX_THREADS, 2>, smem);
                    k_intt<MAXB, NTT_MAX_THREADS, 2><<<total, ntt_threads(p->N), smem, s>>>(B, kp);
                }
                check_launch("k_intt");
            }
        }
    }
}

// Runs the four stages over a list of layers.  Layers of one MAC variant share a launch.
void run_layers(const he_params* p, const KP& kp, const std::vector<StageLayer>& layers, cudaStream_t s, bool timed,
                bool do_mac = true, const cudaEvent_t* marks = nullptr, const cudaEvent_t* input_ready = nullptr) {
    // marks (optional): five events recorded at the stage boundaries
    // input_ready (optional): one event per layer; the input NTTs then run layer by layer, each
    // after its own event (its input's copy), so that they overlap the copies of the later inputs
    auto mark = [&](int i) {
        if (marks) CUDA_OK(cudaEventRecord(marks[i], s));
    };
    mark(0);
    std::vector<const StageLayer*> all;
    for (auto& l : layers) all.push_back(&l);
    const bool single = layers.size() == 1;
    auto go = [&](int stage, const std::vector<const StageLayer*>& ls) {
        if (single) launch_stage<1>(p, kp, stage, ls, s);
        else launch_stage<32>(p, kp, stage, ls, s);
    };
    {
        StageTimer t(HE_STAGE_NTT_IN, s, timed);
        if (input_ready) {
            for (size_t i = 0; i < layers.size(); i++) {
                CUDA_OK(cudaStreamWaitEvent(s, input_ready[i], 0));
                launch_stage<1>(p, kp, ST_NTT, {&layers[i]}, s);
            }
        } else {
            go(ST_NTT, all);
        }
    }
    mark(1);
    {
        // the operand-image layers and the others have different key-switch kernels
        StageTimer t(HE_STAGE_KEYSWITCH, s, timed);
        std::vector<const StageLayer*> grp[2];
        for (auto& l : layers)
            if (!l.dev.fused) grp[l.dev.img ? 1 : 0].push_back(&l);
        for (auto& g : grp)
            if (!g.empty()) go(ST_KS, g);
    }
    mark(2);
    if (do_mac) {
        StageTimer t(HE_STAGE_MAC, s, timed);
        std::vector<bool> done(layers.size(), false);
        for (size_t i = 0; i < layers.size(); i++) {
            if (done[i]) continue;
            std::vector<const StageLayer*> grp;
            for (size_t j = i; j < layers.size(); j++)
                if (!done[j] && layers[j].mv == layers[i].mv) grp.push_back(&layers[j]), done[j] = true;
            go(ST_MAC, grp);
        }
    }
    mark(3);
    {
        StageTimer t(HE_STAGE_NTT_OUT, s, timed);
        go(ST_INTT, all);
    }
    mark(4);
}

}  // namespace

// ================================================================== device tables
namespace hy {
const DeviceTables& device_tables(const he_params* p) {
    int dev = 0;
    CUDA_OK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(p->dev_mu);
    for (DeviceTables* t : p->dev)
        if (t->device == dev) return *t;
    auto T = std::make_unique<DeviceTables>();
    T->device = dev;
    const size_t n = (size_t)p->L * p->N;
    // twiddle and Shoup companion side by side: [L][N][2]
    std::vector<u64> tw(2 * n), itw(2 * n);
    for (u32 k = 0; k < p->L; k++)
        for (u32 i = 0; i < p->N; i++) {
            const size_t o = 2 * ((size_t)k * p->N + i);
            tw[o] = p->ntt[k].tw[i], tw[o + 1] = p->ntt[k].tw_sh[i];
            itw[o] = p->ntt[k].itw[i], itw[o + 1] = p->ntt[k].itw_sh[i];
        }
    u64** dst[2] = {&T->tw, &T->itw};
    std::vector<u64>* srcs[2] = {&tw, &itw};
    for (int i = 0; i < 2; i++) {
        CUDA_OK(cudaMalloc(dst[i], 2 * n * 8));
        CUDA_OK(cudaMemcpy(*dst[i], srcs[i]->data(), 2 * n * 8, cudaMemcpyHostToDevice));
    }
    p->dev.push_back(T.release());
    return *p->dev.back();
}
}  // namespace hy

he_params::~he_params() {
    for (DeviceTables* t : dev) {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess) {
            cudaSetDevice(t->device);
            cudaFree(t->tw);
            cudaFree(t->itw);
            cudaSetDevice(cur);
        }
        delete t;
    }
}

// ================================================================== plan
struct he_plan {
    const he_params* p = nullptr;
    he_conv_desc d{};
    he_layout lay{};
    int device = 0;
    u32 n_rot = 0, rot_id = 0, K = 0, n_ks = 0;
    bool packed = false, h4 = false, dw = false;
    u32 mac_groups = 8;
    bool use_tc = false, eager = false, img = false, fused = false, pair = false, cp = false;
    u32 tc_rows = 0, tc_rows_per_cta = 0, tc_kpad = 0, in_pad = 0, cl = 1;
    u64* d_ksk = nullptr;
    RotDev* d_rots = nullptr;
    RotDev* d_rots_all = nullptr;
    int16_t* d_scal = nullptr;
    u64* d_pk = nullptr;
    u64* d_pksh = nullptr;
    __half* d_sc16 = nullptr;
    int* d_bias = nullptr;
    int* d_err = nullptr;
    u32 tmem_cols = 0, r_slots = 0, r_id = 0;
    size_t off_R = 0, off_D = 0, off_O = 0, off_A = 0, ws_bytes = 0;
    KP kp{};
    ~he_plan() {
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) return;
        cudaSetDevice(device);
        cudaFree(d_ksk);
        cudaFree(d_rots);
        cudaFree(d_rots_all);
        cudaFree(d_scal);
        cudaFree(d_pk);
        cudaFree(d_pksh);
        cudaFree(d_sc16);
        cudaFree(d_bias);
        cudaFree(d_err);
        cudaSetDevice(cur);
    }
    // the stage-layer descriptor of one call
    StageLayer stage_layer(const u64* in, u64* out, char* ws) const {
        StageLayer s;
        std::memset(&s.dev, 0, sizeof(s.dev));
        LayerDev& L = s.dev;
        L.in = in, L.out = out;
        L.R = (u64*)(ws + off_R), L.D = (u64*)(ws + off_D), L.O = (u64*)(ws + off_O);
        L.isrc = L.O;
        L.isrc_stride = 2ull * p->L * p->N;
        L.ksk = d_ksk, L.rots = d_rots, L.scal = d_scal, L.pk = d_pk, L.pksh = d_pksh, L.sc16 = d_sc16, L.bias = d_bias, L.err = d_err;
        L.n_ct_in = lay.n_ct_in, L.n_ct_out = lay.n_ct_out, L.n_rot = n_rot, L.rot_id = rot_id, L.n_ks = n_ks;
        L.K = K, L.Kpad = tc_kpad, L.in_groups = lay.in_groups, L.out_groups = lay.out_groups;
        L.row_units = lay.row_units, L.tc_rows = tc_rows, L.tc_rows_per_cta = tc_rows_per_cta;
        L.tmem_cols = tmem_cols, L.r_slots = r_slots, L.r_id = r_id;
        L.img = img, L.in_pad = in_pad, L.n_rot_all = n_rot, L.id_rot = rot_id, L.rots_all = d_rots_all;
        L.ks_rg = img ? ksi_groups(lay.row_units, in_pad, n_rot, p->L, p->N) : 1;
        L.A16 = img ? (__half*)(ws + off_A) : nullptr;
        if (use_tc && !img) encode_rmap(&L.rmap, L.R, p->N, p->L, lay.n_ct_in * n_rot);
        if (pair) {
            const u64 ktiles = tc_kpad / TC_KTILE, npairs = (tc_rows + 2 * TCP_ROWS - 1) / (2 * TCP_ROWS);
            tcp_encode_maps(&L.rmap, &L.smap, L.A16, (u64)lay.row_units * 2 * p->L * (p->N / TC_MTILE) * ktiles,
                            d_sc16, 2 * npairs * ktiles);
        }
        s.mv.tc = use_tc, s.mv.packed = packed, s.mv.h4 = h4, s.mv.dw = dw, s.mv.eager = eager;
        // groups per CUDA-core MAC block: as many as the kernel holds accumulators for (16 rows)
        s.mv.gt = dw ? 1 : std::min(mac_groups, h4 ? 4u : (packed ? 8u : 16u));
        s.mv.img = img, s.mv.cl = cl, s.mv.fused = fused, s.mv.pair = pair, s.mv.cp = cp;
        L.fused = fused;
        if (fused) L.A16 = nullptr;
        return s;
    }
};

// Builds a plan.  gk == nullptr: timing plan, whose key-switching keys are
// uniform residues made on the device (same sizes and kernels, no secret).
static std::unique_ptr<he_plan> build_plan(const he_params* p, const he_galkeys* gk, const he_conv_desc* d,
                                           const int32_t* weights, const he_tune* tune, bool host_only = false) {
    NvtxRange r("he_conv_plan");
    auto P = std::make_unique<he_plan>();
    P->p = p;
    P->d = *d;
    compute_layout(p, d, &P->lay);
    const he_layout& lay = P->lay;
    P->packed = d->c_n == 2;
    P->h4 = d->c_n == 4;
    P->dw = d->depthwise != 0;
    std::vector<RotEntry> rl = rotation_list(p, d, lay);
    P->n_rot = (u32)rl.size();
    const u32 taps = d->kh * d->kh;
    // rotations that need a key switch, grouped by distinct Galois element
    std::vector<u32> gal;
    std::vector<RotDev> rots, rots_all;
    bool have_id = false;
    for (u32 r = 0; r < rl.size(); r++) {
        if (rl[r].galois == 1) {
            P->rot_id = r;
            have_id = true;
            rots_all.push_back({1u, r, ~0u, 1u});
            continue;
        }
        auto it = std::find(gal.begin(), gal.end(), rl[r].galois);
        u32 key = (u32)(it - gal.begin());
        if (it == gal.end()) gal.push_back(rl[r].galois);
        rots.push_back({rl[r].galois, r, key, galois_inverse(rl[r].galois, p->N)});
        rots_all.push_back(rots.back());
    }
    if (!have_id) fail(HE_EINVAL, "internal: identity rotation missing");
    std::vector<const std::vector<u64>*> keys;
    for (u32 g : gal) {
        if (!gk) break;
        const std::vector<u64>* k = gk->find(g);
        if (!k) fail(HE_EMISSINGKEY, "missing Galois key " + std::to_string(g));
        keys.push_back(k);
    }
    if (p->L * p->l > 16) fail(HE_EINVAL, "L * l must be at most 16");
    // Hadamard scalars s0 = v0 + v1, s1 = v0 - v1 (Eq. 1 without the 1/2); with c_n = 4, s_b = H4 v
    const u32 NR = P->h4 ? 4 : (P->packed ? 2 : 1);
    // a depthwise output reads its own channel's input ciphertext, or with polyphase packing the
    // ciphertexts of its channel's four phase planes (input groups phase-major: phase * out_groups + g)
    const u32 phases = d->polyphase ? 4 : 1;
    P->K = P->dw ? phases * P->n_rot : lay.in_groups * P->n_rot;
    if (P->K > (1u << 14)) fail(HE_EINVAL, "too many accumulation terms (C_in kh^2 > 16384)");
    {
        // every stage of the layer must fit one launch (grid x < 2^31) and 32-bit block indices
        const u64 L = p->L, Nn = p->N, limit = (1ull << 31) - 1;
        const u64 ntt = (u64)lay.n_ct_in * (2 * L + L * p->l * L), intt = (u64)lay.n_ct_out * 2 * L;
        const u64 ks = (u64)rl.size() * L * (Nn / 256);
        const u64 mac = (u64)lay.row_units * 2 * L * (Nn / 128) * lay.out_groups;  // the largest MAC grid
        if (ntt > limit || intt > limit || ks > limit || mac > limit)
            fail(HE_EINVAL, "layer too large for one launch per stage: split its images into several layers");
    }
    std::vector<int16_t> sc((size_t)lay.out_groups * NR * P->K, 0);
    const u32 wcin = P->dw ? 1 : d->C_in;
    // weight of output channel o, input channel i and tap; with polyphase packing i is a plane
    // channel (phase (a, b) = i / Cp, channel i % Cp) and the 3x3 tap (dy', dx') of the derived
    // stride-1 layer is tap (2 dy' + a, 2 dx' + b) of the layer, zero where that lies outside the kernel
    const u32 Cp = (d->C_in + d->c_n - 1) / d->c_n * d->c_n;
    auto W = [&](u32 o, u32 i, u32 tap) -> i64 {
        if (d->polyphase) {
            const u32 ph = i / Cp, c = i % Cp;
            const int dy = 2 * ((int)(tap / 3) - 1) + (int)(ph >> 1), dx = 2 * ((int)(tap % 3) - 1) + (int)(ph & 1);
            if (ph >= 4 || dy < -1 || dy > 1 || dx < -1 || dx > 1) return 0;
            i = c;
            tap = (u32)((dy + 1) * 3 + (dx + 1));
        }
        if (o >= d->C_out || i >= d->C_in) return 0;
        if (P->dw) return o == i ? weights[(size_t)o * taps + tap] : 0;
        return weights[((size_t)o * wcin + i) * taps + tap];
    };
    // c_n = 4: tap index of a block offset dy W_b + dx (unique since W_b > 2P), or none
    std::vector<std::pair<i64, u32>> tap_at;
    for (int dy = -(int)lay.P; dy <= (int)lay.P; dy++)
        for (int dx = -(int)lay.P; dx <= (int)lay.P; dx++)
            tap_at.push_back({(i64)dy * lay.W_b + dx, (u32)((dy + (int)lay.P) * d->kh + dx + (int)lay.P)});
    static const int H4_BASIS[4][4] = {{1, 1, 1, 1}, {1, -1, 1, -1}, {1, 1, -1, -1}, {1, -1, -1, 1}};
    double worst0 = 0, worst1 = 0, worst_abs = 0, worst4[4] = {0, 0, 0, 0};
    for (u32 g = 0; g < lay.out_groups; g++) {
        double s0q = 0, s1q = 0, sab = 0, sq4[4] = {0, 0, 0, 0};
        for (u32 kk = 0; kk < P->K; kk++) {
            u32 j = P->dw ? (kk / P->n_rot) * lay.out_groups + g : kk / P->n_rot, r = kk % P->n_rot;
            u32 tap = rl[r].tap, dg = rl[r].d;
            i64 s0, s1 = 0;
            if (P->h4) {
                // output class c = 2 row + parity e reads, through the copy (step, d), row
                // (c >> 1) ^ d at parity e' = (e + step) mod 2 from offset (e + step - e') / 2
                i64 v[4] = {0, 0, 0, 0};
                for (u32 c = 0; c < 4; c++) {
                    const i64 e = c & 1, es = (e + rl[r].step) & 1, o = (e + rl[r].step - es) / 2;
                    for (auto& ta : tap_at)
                        if (ta.first == o) v[c] = W(4 * g + c, 4 * j + 2 * ((c >> 1) ^ dg) + (u32)es, ta.second);
                }
                for (u32 b = 0; b < 4; b++) {
                    i64 sb = 0;
                    for (u32 c = 0; c < 4; c++) sb += H4_BASIS[b][c] * v[c];
                    if (sb < -32768 || sb > 32767) fail(HE_EINVAL, "weights must satisfy |w| <= 8191 with c_n = 4");
                    sc[((size_t)g * NR + b) * P->K + kk] = (int16_t)sb;
                    sq4[b] += (double)sb * sb, sab += std::fabs((double)sb);
                }
                continue;
            }
            if (P->packed) {
                i64 v0 = dg == 0 ? W(2 * g, 2 * j, tap) : W(2 * g, 2 * j + 1, tap);
                i64 v1 = dg == 0 ? W(2 * g + 1, 2 * j + 1, tap) : W(2 * g + 1, 2 * j, tap);
                s0 = v0 + v1, s1 = v0 - v1;
            } else {
                s0 = W(g, j, tap);
            }
            if (s0 < -32768 || s0 > 32767 || s1 < -32768 || s1 > 32767)
                fail(HE_EINVAL, "weights must satisfy |w| <= 16383");
            sc[((size_t)g * NR + 0) * P->K + kk] = (int16_t)s0;
            if (P->packed) sc[((size_t)g * NR + 1) * P->K + kk] = (int16_t)s1;
            s0q += (double)s0 * s0, s1q += (double)s1 * s1, sab += std::fabs((double)s0) + std::fabs((double)s1);
        }
        worst0 = std::max(worst0, s0q), worst1 = std::max(worst1, s1q), worst_abs = std::max(worst_abs, sab);
        for (u32 b = 0; b < 4; b++) worst4[b] = std::max(worst4[b], sq4[b]);
    }
    double est = P->h4 ? estimate_noise_log2_h4(p, p->w, worst4, worst_abs)
                       : estimate_noise_log2(p, p->w, worst0, worst1, worst_abs, P->packed);
    if (est >= p->log2_delta - 1.0) fail(HE_ENOISE, "estimated noise exceeds Delta/2 for this layer");
    // tensor-core contraction: exact while |s| <= 16 (fp32 sums of 2048-term segments below 2^24)
    int max_abs_s = 0;
    for (int16_t v : sc) max_abs_s = std::max(max_abs_s, std::abs((int)v));
    const u32 impl = tune ? tune->mac_impl : 0;
    // five 10-bit chunks carry a residue only while every limb is below 2^50
    bool limbs_fit = true;
    for (u64 qi : p->q) limbs_fit = limbs_fit && qi < (1ull << (10 * TC_CHUNKS));
    if (P->h4 && impl != 0 && impl != 1)
        fail(HE_EINVAL, "c_n = 4 runs on the CUDA-core MAC only (mac_impl 0 or 1)");
    const bool tc_ok = !P->dw && !P->h4 && max_abs_s <= TC_SMAX && limbs_fit;
    if ((impl == 2 || impl >= 4) && !tc_ok)
        fail(HE_EINVAL, "tensor-core MAC needs |s| <= 16, limbs below 2^50 and a non-depthwise layer");
    if (impl == 3 && P->dw) fail(HE_EINVAL, "the eager MAC is not built for depthwise layers");
    if (impl > 8) fail(HE_EINVAL, "mac_impl must be 0..8");
    if (tune && tune->tc_cluster && tune->tc_cluster != 2 && tune->tc_cluster != 4 && tune->tc_cluster != 8)
        fail(HE_EINVAL, "tc_cluster must be 0, 2, 4 or 8");
    P->eager = impl == 3;
    P->use_tc = tc_ok && impl != 1 && impl != 3;
    P->in_pad = (lay.in_groups + 7) / 8 * 8;
    if (tune && tune->mac_groups) {
        const u32 mg = tune->mac_groups;
        if (mg > 16 || (mg & (mg - 1))) fail(HE_EINVAL, "mac_groups must be 1, 2, 4, 8 or 16");
        P->mac_groups = mg;
    }
    const u32 tc_rows_req = tune ? tune->tc_rows : 0;
    if (tc_rows_req && (tc_rows_req % 16 || tc_rows_req > (u32)TC_NMAX))
        fail(HE_EINVAL, "tc_rows must be a multiple of 16, at most 96");
    if (P->use_tc) {
        const u32 rows = lay.out_groups * NR;
        P->tc_rows = (rows + 15) / 16 * 16;
        P->tc_rows_per_cta = std::min<u32>(tc_rows_req ? tc_rows_req : TC_NMAX, P->tc_rows);
        // the form of the contraction, from per-layer timings of the ResNet-20, VGG-16 and
        // MobileNetV1 stacks: operand images written once by the key switch (5) unless the layer's
        // rows fit one CTA (no row tile would split the residues again) and either the image form
        // would pad the input channel groups (first layers: 3 channels) or the digit transforms
        // of all input ciphertexts fit in L2 (the word-form key switch then reuses them well); those
        // take the key switch's words and split them in the MAC (4).  6 runs the key switch in the MAC.
        const bool one_tile = P->tc_rows <= P->tc_rows_per_cta;
        const size_t digit_bytes = (size_t)lay.n_ct_in * (p->L * p->l * p->L + 2 * p->L) * p->N * 8;
        const bool words = one_tile && (P->in_pad != lay.in_groups || digit_bytes <= (64u << 20));
        const u32 form = (impl >= 4) ? impl : (words ? 4u : 5u);
        if (form == 6 && (!one_tile || (tune && tune->tc_cluster)))
            fail(HE_EINVAL, "the fused key switch + MAC needs a layer whose rows fit one CTA and no cluster");
        if (form >= 7 && ((tune && tune->tc_cluster) || tc_rows_req))
            fail(HE_EINVAL, "the CTA-pair and chunk-pass MACs take no tc_rows and no tc_cluster");
        P->img = form != 4;
        P->fused = form == 6;
        P->pair = form == 7;
        P->cp = form == 8;
        if (P->pair) P->tc_rows_per_cta = TCP_ROWS;
        if (P->cp) P->tc_rows_per_cta = std::min<u32>(TCC_ROWS, P->tc_rows);
        P->cl = 1;
        const u32 cl_req = tune ? tune->tc_cluster : 0;
        if (cl_req > 1) {
            // clusters of cl_req CTAs share each operand image by multicast: the row tiles of a slot
            // tile are split into a multiple of cl_req tiles of at most 96 rows, none of them empty
            const u32 m = cl_req * ((P->tc_rows + TC_NMAX * cl_req - 1) / (TC_NMAX * cl_req));
            const u32 rpc = ((P->tc_rows + m - 1) / m + 15) / 16 * 16;
            if (!P->img || P->fused || P->pair || P->cp || tc_rows_req || P->tc_rows <= (m - 1) * rpc)
                fail(HE_EINVAL, "tc_cluster needs the image-form tensor-core MAC, no tc_rows, and at least " +
                                    std::to_string(16 * (m - 1) + 16) + " output rows");
            P->cl = cl_req, P->tc_rows_per_cta = rpc;
        }
    }
    if (host_only) return P;
    // device data
    CUDA_OK(cudaGetDevice(&P->device));
    P->kp = make_kp(p);
    cudaStream_t s = 0;
    if (gk) {
        P->d_ksk = upload_keys(p, P->kp, keys, s);
    } else if (!gal.empty()) {
        const size_t per = (size_t)p->L * p->l * 2 * p->L * p->N;
        CUDA_OK(cudaMalloc(&P->d_ksk, per * gal.size() * 8));
        fill_uniform(P->kp, P->d_ksk, per * gal.size() / p->N, 0x5eed, s);
    }
    P->n_ks = (u32)rots.size();
    if (!rots.empty()) {
        CUDA_OK(cudaMalloc(&P->d_rots, rots.size() * sizeof(RotDev)));
        CUDA_OK(cudaMemcpy(P->d_rots, rots.data(), rots.size() * sizeof(RotDev), cudaMemcpyHostToDevice));
    }
    CUDA_OK(cudaMalloc(&P->d_rots_all, rots_all.size() * sizeof(RotDev)));
    CUDA_OK(cudaMemcpy(P->d_rots_all, rots_all.data(), rots_all.size() * sizeof(RotDev), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMalloc(&P->d_scal, sc.size() * sizeof(int16_t)));
    CUDA_OK(cudaMemcpy(P->d_scal, sc.data(), sc.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
    // NTT(P_k): P_k = kh (X^(N/4) + X^(3N/4)) lifted into every limb; with c_n = 4 the three
    // k4-scaled patterns [3][L][N], their centred coefficients lifted the same way
    if (P->packed || P->h4) {
        const u32 nb = P->h4 ? 3 : 1;
        std::vector<u64> pk((size_t)nb * p->L * p->N, 0);
        for (u32 b = 0; b < nb; b++)
            for (u32 k = 0; k < p->L; k++) {
                u64* row = pk.data() + ((size_t)b * p->L + k) * p->N;
                if (P->h4) {
                    for (u32 j = 0; j < p->N; j++) {
                        const i64 a = p->pat4[(size_t)b * p->N + j];
                        if (!a) continue;
                        i64 v = (i64)(((__int128)a * (i64)p->k4) % (i64)p->t);
                        if (v > (i64)(p->t / 2)) v -= (i64)p->t;
                        if (v < -(i64)(p->t / 2)) v += (i64)p->t;
                        row[j] = p->mod[k].from_signed(v);
                    }
                } else {
                    const u64 v = p->mod[k].from_signed(p->kh);
                    row[p->N / 4] = v;
                    row[3 * p->N / 4] = v;
                }
                p->ntt[k].forward(row);
            }
        CUDA_OK(cudaMalloc(&P->d_pk, pk.size() * 8));
        CUDA_OK(cudaMemcpy(P->d_pk, pk.data(), pk.size() * 8, cudaMemcpyHostToDevice));
        std::vector<u64> pksh(pk.size());
        for (size_t i = 0; i < pk.size(); i++) {
            const u64 q = p->q[(i / p->N) % p->L];
            pksh[i] = (u64)((((unsigned __int128)pk[i]) << 64) / q);
        }
        CUDA_OK(cudaMalloc(&P->d_pksh, pksh.size() * 8));
        CUDA_OK(cudaMemcpy(P->d_pksh, pksh.data(), pksh.size() * 8, cudaMemcpyHostToDevice));
    }
    CUDA_OK(cudaMalloc(&P->d_err, sizeof(int)));
    CUDA_OK(cudaMemset(P->d_err, 0, sizeof(int)));
    if (P->use_tc) {
        // terms: kk = j n_rot + rot for the in-kernel conversion form, rot in_pad + j for the image form
        const u32 k_terms = P->img ? P->n_rot * P->in_pad : P->K;
        P->tc_kpad = (k_terms + TC_KTILE - 1) / TC_KTILE * TC_KTILE;
        // scalar tiles stored as the exact shared-memory image the MMA reads (K-major, no
        // swizzle), one block of rows_per_cta x 32 terms per (row tile, K tile); the CTA-pair form
        // has two tiles of 128 rows per pair tile, each ordered diagonal-major (see k_mac_pair)
        const u32 rpc = P->tc_rows_per_cta, ktiles = P->tc_kpad / TC_KTILE;
        const u32 mtiles = P->pair ? 2 * ((P->tc_rows + 2 * TCP_ROWS - 1) / (2 * TCP_ROWS)) : (P->tc_rows + rpc - 1) / rpc;
        std::vector<__half> h16((size_t)mtiles * ktiles * rpc * TC_KTILE, __float2half(0.0f));
        // bias [segment][row] = 512 x the sum of the row's scalars over the segment's terms
        const u32 n_seg = (ktiles + TC_SEG_TILES - 1) / TC_SEG_TILES;
        std::vector<int> bias((size_t)n_seg * P->tc_rows, 0);
        for (u32 g = 0; g < lay.out_groups; g++)
            for (u32 r = 0; r < NR; r++) {
                const u32 row = g * NR + r, per = P->packed ? TCP_ROWS / 2 : TCP_ROWS;
                const u32 mt = P->pair ? g / per : row / rpc, rl = P->pair ? r * (TCP_ROWS / 2) + g % per : row % rpc;
                for (u32 kk0 = 0; kk0 < P->K; kk0++) {
                    int v = sc[((size_t)g * NR + r) * P->K + kk0];
                    const u32 kk = P->img ? (kk0 % P->n_rot) * P->in_pad + kk0 / P->n_rot : kk0;
                    const u32 kt = kk / TC_KTILE, kl = kk % TC_KTILE;
                    const size_t byte = ((size_t)mt * ktiles + kt) * rpc * TC_KTILE * 2 +
                                        (rl >> 3) * TC_SBO + (kl >> 3) * 128 + (rl & 7) * 16 + (kl & 7) * 2;
                    h16[byte / 2] = __float2half((float)v);
                    bias[(size_t)(kt / TC_SEG_TILES) * P->tc_rows + row] += 512 * v;
                }
            }
        CUDA_OK(cudaMalloc(&P->d_sc16, h16.size() * sizeof(__half)));
        CUDA_OK(cudaMemcpy(P->d_sc16, h16.data(), h16.size() * sizeof(__half), cudaMemcpyHostToDevice));
        CUDA_OK(cudaMalloc(&P->d_bias, bias.size() * sizeof(int)));
        CUDA_OK(cudaMemcpy(P->d_bias, bias.data(), bias.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    if (P->use_tc) {
        u32 cols = 32;
        while (cols < (u32)TC_CHUNKS * P->tc_rows_per_cta) cols <<= 1;
        P->tmem_cols = (P->pair || P->cp) ? 512 : cols;  // the pair form holds 5 x 64 columns, chunk passes all 512
    }
    CUDA_OK(cudaStreamSynchronize(s));
    // workspace: R [n_ct_in][r_slots][2][L][N], D [n_ct_in][L l][L][N], O [n_ct_out][2][L][N] and, for
    // the image form, A [row_units][2][L][N/128][Kpad/32] operand images of 40 KB (R then holds only
    // the identity rotation, NTT(c0) and NTT(c1))
    P->r_slots = P->img ? 1 : P->n_rot;
    P->r_id = P->img ? 0 : P->rot_id;
    const size_t ctw = 2ull * p->L * p->N;
    P->off_R = 0;
    P->off_D = align256(P->off_R + (size_t)lay.n_ct_in * P->r_slots * ctw * 8);
    P->off_O = align256(P->off_D + (size_t)lay.n_ct_in * p->L * p->l * p->L * p->N * 8);
    P->off_A = align256(P->off_O + (size_t)lay.n_ct_out * ctw * 8);
    const size_t img_bytes = P->img && !P->fused ? (size_t)lay.row_units * 2 * p->L * (p->N / TC_MTILE) *
                                                       (P->tc_kpad / TC_KTILE) * IMG_HALVES * 2
                                                 : 0;
    P->ws_bytes = align256(P->off_A + img_bytes);
    (void)taps;
    return P;
}

extern "C" int he_conv_plan(const he_params* p, const he_galkeys* gk, const he_conv_desc* d, const int32_t* weights,
                            const he_tune* tune, he_plan** out) {
    return guard([&] {
        if (!p || !gk || !d || !weights || !out) fail(HE_EINVAL, "null argument");
        if (gk->p != p) fail(HE_EINVAL, "Galois keys belong to other parameters");
        *out = nullptr;
        *out = build_plan(p, gk, d, weights, tune).release();
    });
}

extern "C" int he_conv_sizes(const he_plan* plan, size_t* in_words, size_t* out_words, size_t* ws) {
    return guard([&] {
        if (!plan) fail(HE_EINVAL, "null plan");
        const size_t ctw = 2ull * plan->p->L * plan->p->N;
        if (in_words) *in_words = plan->lay.n_ct_in * ctw;
        if (out_words) *out_words = plan->lay.n_ct_out * ctw;
        if (ws) *ws = plan->ws_bytes;
    });
}

static void check_ptrs(const void* a, const void* b, const void* c) {
    if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15) fail(HE_EINVAL, "device pointers must be 16-byte aligned");
}
static void check_device(int device) {
    int dev = -1;
    CUDA_OK(cudaGetDevice(&dev));
    if (dev != device) fail(HE_EINVAL, "plan was made on another device");
}

static void forward_impl(const he_plan* P, const u64* d_in, u64* d_out, void* ws, cudaStream_t s, bool timed = true) {
    NvtxRange r("he_conv_forward");
    check_ptrs(d_in, d_out, ws);
    check_device(P->device);
    std::vector<StageLayer> ls{P->stage_layer(d_in, d_out, (char*)ws)};
    run_layers(P->p, P->kp, ls, s, timed);
}

extern "C" int he_conv_forward(const he_plan* plan, const uint64_t* d_in, uint64_t* d_out, void* d_ws, void* stream) {
    return guard([&] {
        if (!plan || !d_in || !d_out || !d_ws) fail(HE_EINVAL, "null argument");
        forward_impl(plan, d_in, d_out, d_ws, (cudaStream_t)stream);
    });
}

extern "C" int he_conv_forward_host(const he_plan* plan, const uint64_t* h_in, uint64_t* h_out, uint64_t* d_in,
                                    uint64_t* d_out, void* d_ws, void* stream) {
    return guard([&] {
        if (!plan || !h_in || !h_out || !d_in || !d_out || !d_ws) fail(HE_EINVAL, "null argument");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t ctw = 2ull * plan->p->L * plan->p->N;
        CUDA_OK(cudaMemcpyAsync(d_in, h_in, plan->lay.n_ct_in * ctw * 8, cudaMemcpyHostToDevice, s));
        forward_impl(plan, d_in, d_out, d_ws, s);
        CUDA_OK(cudaMemcpyAsync(h_out, d_out, plan->lay.n_ct_out * ctw * 8, cudaMemcpyDeviceToHost, s));
        CUDA_OK(cudaStreamSynchronize(s));
    });
}

extern "C" int he_conv_status(const he_plan* plan) {
    return guard([&] {
        if (!plan) fail(HE_EINVAL, "null plan");
        int v = 0;
        CUDA_OK(cudaMemcpy(&v, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (v) fail(HE_ETIMEOUT, "a bounded device wait in the tensor-core MAC gave up");
    });
}

extern "C" int he_selftest_bounded_wait(void* stream) {
    return guard([&] {
        cudaStream_t s = (cudaStream_t)stream;
        int* d_err = nullptr;
        CUDA_OK(cudaMalloc(&d_err, sizeof(int)));
        struct Free {
            int* p;
            ~Free() { cudaFree(p); }
        } f{d_err};
        CUDA_OK(cudaMemsetAsync(d_err, 0, sizeof(int), s));
        k_wait_selftest<<<1, 32, 0, s>>>(d_err, TC_SPIN_LIMIT >> 6);
        check_launch("k_wait_selftest");
        int v = 0;
        CUDA_OK(cudaMemcpyAsync(&v, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_OK(cudaStreamSynchronize(s));
        if (v) fail(HE_ETIMEOUT, "bounded wait gave up as designed");
    });
}

extern "C" int he_conv_check(const he_params* p, const he_conv_desc* d, const int32_t* weights, const he_tune* tune) {
    return guard([&] {
        if (!p || !d || !weights) fail(HE_EINVAL, "null argument");
        build_plan(p, nullptr, d, weights, tune, true);
    });
}

extern "C" int he_conv_time(const he_params* p, const he_conv_desc* d, const int32_t* weights, const he_tune* tune,
                            int reps, void* stream, float* stage_ms, float* total_ms) {
    return guard([&] {
        if (!p || !d || !weights || !total_ms || reps < 1 || reps > 1000) fail(HE_EINVAL, "bad argument");
        std::unique_ptr<he_plan> P = build_plan(p, nullptr, d, weights, tune);
        cudaStream_t s = (cudaStream_t)stream;
        const size_t ctw = 2ull * p->L * p->N;
        struct Buf {
            void* ptr = nullptr;
            ~Buf() {
                if (ptr) cudaFree(ptr);
            }
        } in, out, ws;
        CUDA_OK(cudaMalloc(&in.ptr, std::max<size_t>(256, P->lay.n_ct_in * ctw * 8)));
        CUDA_OK(cudaMalloc(&out.ptr, std::max<size_t>(256, P->lay.n_ct_out * ctw * 8)));
        CUDA_OK(cudaMalloc(&ws.ptr, std::max<size_t>(256, P->ws_bytes)));
        fill_uniform(P->kp, (u64*)in.ptr, (size_t)P->lay.n_ct_in * 2 * p->L, 0xc0ffee, s);
        struct Events {
            cudaEvent_t e[5] = {};
            ~Events() {
                for (auto x : e)
                    if (x) cudaEventDestroy(x);
            }
        } ev;
        for (auto& x : ev.e) CUDA_OK(cudaEventCreate(&x));
        std::vector<StageLayer> ls{P->stage_layer((const u64*)in.ptr, (u64*)out.ptr, (char*)ws.ptr)};
        run_layers(p, P->kp, ls, s, false);  // warm-up (also sets the kernels' attributes)
        std::vector<std::vector<float>> t(5, std::vector<float>(reps));
        for (int r = 0; r < reps; r++) {
            run_layers(p, P->kp, ls, s, false, true, ev.e);
            CUDA_OK(cudaEventSynchronize(ev.e[4]));
            for (int i = 0; i < 4; i++) CUDA_OK(cudaEventElapsedTime(&t[i][r], ev.e[i], ev.e[i + 1]));
            CUDA_OK(cudaEventElapsedTime(&t[4][r], ev.e[0], ev.e[4]));
        }
        int v = 0;
        CUDA_OK(cudaMemcpy(&v, P->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (v) fail(HE_ETIMEOUT, "a bounded device wait in the tensor-core MAC gave up");
        auto median = [](std::vector<float> x) {
            std::sort(x.begin(), x.end());
            return x[x.size() / 2];
        };
        for (int i = 0; i < 4 && stage_ms; i++) stage_ms[i] = median(t[i]);
        *total_ms = median(t[4]);
    });
}

extern "C" int he_conv_info(const he_plan* plan, int* mac_impl) {
    return guard([&] {
        if (!plan || !mac_impl) fail(HE_EINVAL, "null argument");
        *mac_impl = plan->use_tc ? (plan->cp ? 8 : plan->pair ? 7 : (plan->fused ? 6 : (plan->img ? 5 : 4)))
                                 : (plan->eager ? 3 : 1);
    });
}

extern "C" void he_plan_destroy(he_plan* plan) { delete plan; }

// ================================================================== batches of layers
struct he_batch {
    std::vector<const he_plan*> plans;
    const he_params* p = nullptr;
    int device = 0;
    // layers run in waves that reuse one workspace region; ws_off is a layer's offset inside it
    std::vector<std::vector<u32>> waves;
    std::vector<size_t> ws_off;
    size_t ws_bytes = 0;
    // captured graph and the pointers it was captured with
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> g_in, g_out;
    const void* g_ws = nullptr;
    cudaStream_t g_stream = nullptr;
    // end-to-end form: two halves of a one-wave batch on two streams, so that the copies of one
    // half overlap the kernels of the other (see he_batch_forward_host)
    std::unique_ptr<he_batch> half[2];
    std::vector<u32> half_idx[2];
    cudaStream_t s2 = nullptr, s3 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_done;  // per wave: inputs copied, kernels done
    std::vector<cudaEvent_t> ev_first;        // per layer of the first wave: its input copied
    ~he_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (auto e : ev_in) cudaEventDestroy(e);
        for (auto e : ev_first) cudaEventDestroy(e);
        for (auto e : ev_done) cudaEventDestroy(e);
        if (s2) cudaStreamDestroy(s2);
        if (s3) cudaStreamDestroy(s3);
    }
    std::vector<StageLayer> layers(const std::vector<u32>& wave, const uint64_t* const* d_in, uint64_t* const* d_out,
                                   char* ws) const {
        std::vector<StageLayer> ls;
        for (u32 i : wave) ls.push_back(plans[i]->stage_layer(d_in[i], d_out[i], ws + ws_off[i]));
        return ls;
    }
    void run(const uint64_t* const* d_in, uint64_t* const* d_out, char* ws, cudaStream_t s, bool timed) const {
        NvtxRange r("he_batch");
        for (const auto& w : waves) run_layers(p, plans[0]->kp, layers(w, d_in, d_out, ws), s, timed);
    }
};

extern "C" int he_batch_create_limited(const he_plan* const* plans, int n, size_t max_workspace_bytes,
                                       he_batch** out) {
    return guard([&] {
        if (!plans || n <= 0 || !out) fail(HE_EINVAL, "bad argument");
        auto B = std::make_unique<he_batch>();
        B->p = plans[0]->p;
        B->device = plans[0]->device;
        for (int i = 0; i < n; i++) {
            if (!plans[i]) fail(HE_EINVAL, "null plan");
            if (plans[i]->p != B->p) fail(HE_EINVAL, "all plans of a batch must share their parameters");
            if (plans[i]->device != B->device) fail(HE_EINVAL, "all plans of a batch must be on one device");
            B->plans.push_back(plans[i]);
        }
        // first fit, largest workspace first; a layer larger than the limit gets a wave of its own
        std::vector<u32> order(n);
        for (int i = 0; i < n; i++) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](u32 a, u32 b) { return plans[a]->ws_bytes > plans[b]->ws_bytes; });
        std::vector<size_t> used;
        B->ws_off.assign(n, 0);
        for (u32 i : order) {
            const size_t need = align256(plans[i]->ws_bytes);
            size_t w = 0;
            while (w < used.size() && used[w] + need > max_workspace_bytes) w++;
            if (w == used.size()) used.push_back(0), B->waves.emplace_back();
            B->ws_off[i] = used[w];
            used[w] += need;
            B->waves[w].push_back(i);
        }
        // layers of a wave in their given order
        for (auto& w : B->waves) std::sort(w.begin(), w.end());
        for (size_t u : used) B->ws_bytes = std::max(B->ws_bytes, u);
        *out = B.release();
    });
}

extern "C" int he_batch_create(const he_plan* const* plans, int n, he_batch** out) {
    return he_batch_create_limited(plans, n, SIZE_MAX, out);
}

extern "C" int he_batch_waves(const he_batch* b, int* n_waves) {
    return guard([&] {
        if (!b || !n_waves) fail(HE_EINVAL, "null argument");
        *n_waves = (int)b->waves.size();
    });
}

extern "C" int he_batch_workspace_bytes(const he_batch* b, size_t* bytes) {
    return guard([&] {
        if (!b || !bytes) fail(HE_EINVAL, "null argument");
        *bytes = b->ws_bytes;
    });
}

extern "C" int he_batch_forward(const he_batch* b, const uint64_t* const* d_in, uint64_t* const* d_out, void* d_ws,
                                void* stream) {
    return guard([&] {
        if (!b || !d_in || !d_out || !d_ws) fail(HE_EINVAL, "null argument");
        check_device(b->device);
        for (size_t i = 0; i < b->plans.size(); i++) check_ptrs(d_in[i], d_out[i], d_ws);
        b->run(d_in, d_out, (char*)d_ws, (cudaStream_t)stream, true);
    });
}

static void batch_graph_launch(he_batch* b, const uint64_t* const* d_in, uint64_t* const* d_out, void* d_ws,
                               cudaStream_t s) {
    check_device(b->device);
    bool same = b->exec && b->g_ws == d_ws && b->g_stream == s;
    for (size_t i = 0; same && i < b->plans.size(); i++) same = b->g_in[i] == d_in[i] && b->g_out[i] == d_out[i];
    if (!same) {
        for (size_t i = 0; i < b->plans.size(); i++) check_ptrs(d_in[i], d_out[i], d_ws);
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        // one ordinary pass sets the kernels' attributes before capture
        b->run(d_in, d_out, (char*)d_ws, s, false);
        cudaGraph_t g = nullptr;
        CUDA_OK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            b->run(d_in, d_out, (char*)d_ws, s, false);
        } catch (...) {
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        CUDA_OK(cudaStreamEndCapture(s, &g));
        cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) fail(HE_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        b->g_in.assign(d_in, d_in + b->plans.size());
        b->g_out.assign(d_out, d_out + b->plans.size());
        b->g_ws = d_ws;
        b->g_stream = s;
    }
    CUDA_OK(cudaGraphLaunch(b->exec, s));
}

extern "C" int he_batch_graph_launch(he_batch* b, const uint64_t* const* d_in, uint64_t* const* d_out, void* d_ws,
                                     void* stream) {
    return guard([&] {
        if (!b || !d_in || !d_out || !d_ws || !stream) fail(HE_EINVAL, "graph launches need pointers and a non-default stream");
        batch_graph_launch(b, d_in, d_out, d_ws, (cudaStream_t)stream);
    });
}

// Splits a one-wave batch into two halves of about equal input size (layers keep their workspace
// offsets, so the halves can run at the same time), each with its own graph.
static void make_halves(he_batch* b) {
    const size_t ctw = 2ull * b->p->L * b->p->N;
    size_t total = 0, acc = 0;
    for (auto* pl : b->plans) total += pl->lay.n_ct_in * ctw;
    for (u32 i = 0; i < b->plans.size(); i++) {
        const int h = (acc * 2 < total) ? 0 : 1;
        b->half_idx[h].push_back(i);
        acc += b->plans[i]->lay.n_ct_in * ctw;
    }
    if (b->half_idx[1].empty()) {  // one layer holds most of the input: it alone is the second half
        b->half_idx[1].push_back(b->half_idx[0].back());
        b->half_idx[0].pop_back();
    }
    for (int h = 0; h < 2; h++) {
        auto c = std::make_unique<he_batch>();
        c->p = b->p;
        c->device = b->device;
        c->waves.emplace_back();
        for (u32 j = 0; j < b->half_idx[h].size(); j++) {
            const u32 i = b->half_idx[h][j];
            c->plans.push_back(b->plans[i]);
            c->ws_off.push_back(b->ws_off[i]);
            c->waves[0].push_back(j);
        }
        c->ws_bytes = b->ws_bytes;
        b->half[h] = std::move(c);
    }
    CUDA_OK(cudaStreamCreateWithFlags(&b->s2, cudaStreamNonBlocking));
    CUDA_OK(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    CUDA_OK(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
}

extern "C" int he_batch_forward_host(he_batch* b, const uint64_t* const* h_in, uint64_t* const* h_out,
                                     uint64_t* const* d_in, uint64_t* const* d_out, void* d_ws, void* stream) {
    return guard([&] {
        if (!b || !h_in || !h_out || !d_in || !d_out || !d_ws || !stream)
            fail(HE_EINVAL, "null argument (host and device buffers of every layer, a non-default stream)");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t ctw = 2ull * b->p->L * b->p->N;
        for (size_t i = 0; i < b->plans.size(); i++)
            if (!h_in[i] || !h_out[i]) fail(HE_EINVAL, "null host buffer");
        check_device(b->device);
        if (b->plans.size() < 2) {
            CUDA_OK(cudaMemcpyAsync(d_in[0], h_in[0], b->plans[0]->lay.n_ct_in * ctw * 8, cudaMemcpyHostToDevice, s));
            batch_graph_launch(b, d_in, d_out, d_ws, s);
            CUDA_OK(cudaMemcpyAsync(h_out[0], d_out[0], b->plans[0]->lay.n_ct_out * ctw * 8, cudaMemcpyDeviceToHost, s));
            CUDA_OK(cudaStreamSynchronize(s));
            return;
        }
        if (b->waves.size() > 1) {
            // waves run one after another on s (they share the workspace region); the inputs of
            // every wave stream in on s2 ahead of its kernels, the outputs of a finished wave leave
            // on s3 while the next wave computes.  The first wave's input NTTs run layer by layer as
            // their inputs land, so that only the first layer's copy is exposed
            const size_t nw = b->waves.size();
            if (!b->s2) {
                CUDA_OK(cudaStreamCreateWithFlags(&b->s2, cudaStreamNonBlocking));
                CUDA_OK(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
                CUDA_OK(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
            }
            if (!b->s3) CUDA_OK(cudaStreamCreateWithFlags(&b->s3, cudaStreamNonBlocking));
            while (b->ev_in.size() < nw) {
                cudaEvent_t a, c;
                CUDA_OK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
                b->ev_in.push_back(a);
                CUDA_OK(cudaEventCreateWithFlags(&c, cudaEventDisableTiming));
                b->ev_done.push_back(c);
            }
            while (b->ev_first.size() < b->waves[0].size()) {
                cudaEvent_t a;
                CUDA_OK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
                b->ev_first.push_back(a);
            }
            CUDA_OK(cudaEventRecord(b->ev_fork, s));
            CUDA_OK(cudaStreamWaitEvent(b->s2, b->ev_fork, 0));
            CUDA_OK(cudaStreamWaitEvent(b->s3, b->ev_fork, 0));
            for (size_t w = 0; w < nw; w++) {
                for (size_t q = 0; q < b->waves[w].size(); q++) {
                    const u32 i = b->waves[w][q];
                    CUDA_OK(cudaMemcpyAsync(d_in[i], h_in[i], b->plans[i]->lay.n_ct_in * ctw * 8, cudaMemcpyHostToDevice,
                                            b->s2));
                    if (w == 0) CUDA_OK(cudaEventRecord(b->ev_first[q], b->s2));
                }
                CUDA_OK(cudaEventRecord(b->ev_in[w], b->s2));
            }
            for (size_t w = 0; w < nw; w++) {
                if (w > 0) CUDA_OK(cudaStreamWaitEvent(s, b->ev_in[w], 0));
                run_layers(b->p, b->plans[0]->kp, b->layers(b->waves[w], d_in, d_out, (char*)d_ws), s, true, true,
                           nullptr, w == 0 ? b->ev_first.data() : nullptr);
                CUDA_OK(cudaEventRecord(b->ev_done[w], s));
                CUDA_OK(cudaStreamWaitEvent(b->s3, b->ev_done[w], 0));
                for (u32 i : b->waves[w])
                    CUDA_OK(cudaMemcpyAsync(h_out[i], d_out[i], b->plans[i]->lay.n_ct_out * ctw * 8,
                                            cudaMemcpyDeviceToHost, b->s3));
            }
            CUDA_OK(cudaEventRecord(b->ev_join, b->s3));
            CUDA_OK(cudaStreamWaitEvent(s, b->ev_join, 0));
            CUDA_OK(cudaStreamSynchronize(s));
            return;
        }
        if (!b->half[0]) make_halves(b);
        // the second stream starts after the caller's earlier work on s
        CUDA_OK(cudaEventRecord(b->ev_fork, s));
        CUDA_OK(cudaStreamWaitEvent(b->s2, b->ev_fork, 0));
        for (int h = 0; h < 2; h++) {
            cudaStream_t sh = h ? b->s2 : s;
            const auto& idx = b->half_idx[h];
            std::vector<const uint64_t*> di;
            std::vector<uint64_t*> dout;
            for (u32 i : idx) {
                CUDA_OK(cudaMemcpyAsync(d_in[i], h_in[i], b->plans[i]->lay.n_ct_in * ctw * 8, cudaMemcpyHostToDevice, sh));
                di.push_back(d_in[i]);
                dout.push_back(d_out[i]);
            }
            batch_graph_launch(b->half[h].get(), di.data(), dout.data(), d_ws, sh);
            for (u32 i : idx)
                CUDA_OK(cudaMemcpyAsync(h_out[i], d_out[i], b->plans[i]->lay.n_ct_out * ctw * 8, cudaMemcpyDeviceToHost, sh));
        }
        CUDA_OK(cudaEventRecord(b->ev_join, b->s2));
        CUDA_OK(cudaStreamWaitEvent(s, b->ev_join, 0));
        CUDA_OK(cudaStreamSynchronize(s));
    });
}

extern "C" void he_batch_destroy(he_batch* b) { delete b; }

// ================================================================== allocation-free forward
// Scratch for he_conv_forward_noalloc.  A file-scope device array: the CUDA
// runtime reserves it on every device that loads this library, for the life
// of the process, so the entry point itself never allocates.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HE_NOALLOC_MAX_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
std::vector<std::pair<int, void*>> g_noalloc_addr;  // (device, device address of g_noalloc_scratch)

// Device address of the scratch array on the current device.  In host code
// the name g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up once per device with that device current.
void* noalloc_scratch() {
    int dev = -1;
    CUDA_OK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    for (auto& e : g_noalloc_addr)
        if (e.first == dev) return e.second;
    void* ptr = nullptr;
    CUDA_OK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    if (!ptr) fail(HE_ECUDA, "cudaGetSymbolAddress returned a null scratch address");
    g_noalloc_addr.push_back({dev, ptr});
    return ptr;
}
}  // namespace

extern "C" int he_conv_forward_noalloc(const he_plan* plan, const uint64_t* d_in, uint64_t* d_out, void* stream) {
    return guard([&] {
        if (!plan || !d_in || !d_out) fail(HE_EINVAL, "null argument");
        if (plan->ws_bytes > (size_t)HE_NOALLOC_MAX_SCRATCH_BYTES)
            fail(HE_EINVAL, "layer needs " + std::to_string(plan->ws_bytes) + " bytes of scratch; the static scratch holds " +
                                std::to_string((size_t)HE_NOALLOC_MAX_SCRATCH_BYTES) + " (use he_conv_forward)");
        // a call that will be refused touches no device: the plan's device and the caller's
        // pointers are checked before the scratch address is looked up
        check_device(plan->device);
        check_ptrs(d_in, d_out, nullptr);
        void* ws = noalloc_scratch();
        // every scratch word a kernel reads was written earlier in the same call,
        // so nothing has to be cleared between calls
        forward_impl(plan, d_in, d_out, ws, (cudaStream_t)stream, /*timed=*/false);
    });
}

// ================================================================== single steps
extern "C" int he_ntt_forward(const he_params* p, uint64_t* d, int n, void* stream) {
    return guard([&] {
        if (!p || (!d && n > 0) || n < 0) fail(HE_EINVAL, "bad argument");
        KP kp = make_kp(p);
        launch_ntt_plain(p, kp, d, n, 0, (cudaStream_t)stream);
    });
}
extern "C" int he_ntt_inverse(const he_params* p, uint64_t* d, int n, void* stream) {
    return guard([&] {
        if (!p || (!d && n > 0) || n < 0) fail(HE_EINVAL, "bad argument");
        KP kp = make_kp(p);
        launch_ntt_plain(p, kp, d, n, 1, (cudaStream_t)stream);
    });
}

static void rotate_offsets(const he_params* p, int n_ct, size_t* offD, size_t* total) {
    const size_t ctw = 2ull * p->L * p->N;
    *offD = align256((size_t)n_ct * 2 * ctw * 8);
    *total = align256(*offD + (size_t)n_ct * p->L * p->l * p->L * p->N * 8);
}
extern "C" int he_rotate_workspace_bytes(const he_params* p, int n_ct, size_t* bytes) {
    return guard([&] {
        if (!p || !bytes || n_ct < 0) fail(HE_EINVAL, "bad argument");
        size_t offD;
        rotate_offsets(p, n_ct, &offD, bytes);
    });
}
extern "C" int he_rotate(const he_params* p, const he_galkeys* gk, uint32_t galois, const uint64_t* d_in,
                         uint64_t* d_out, int n_ct, void* d_ws, void* stream) {
    return guard([&] {
        if (!p || !gk || !d_in || !d_out || !d_ws || n_ct <= 0) fail(HE_EINVAL, "bad argument");
        const std::vector<u64>* key = gk->find(galois);
        if (!key) fail(HE_EMISSINGKEY, "missing Galois key");
        if (p->L * p->l > 16) fail(HE_EINVAL, "L * l must be at most 16");
        check_ptrs(d_in, d_out, d_ws);
        cudaStream_t s = (cudaStream_t)stream;
        KP kp = make_kp(p);
        // device copies of the key and the rotation record, freed on every path out
        struct Free {
            void* p = nullptr;
            ~Free() {
                if (p) cudaFree(p);
            }
        } fkey, frot;
        u64* dkey = upload_keys(p, kp, {key}, s);
        fkey.p = dkey;
        if (!(galois & 1) || galois >= 2 * p->N) fail(HE_EINVAL, "Galois element must be odd and below 2N");
        RotDev rd{galois, 1, 0, galois_inverse(galois, p->N)};
        RotDev* drot = nullptr;
        CUDA_OK(cudaMalloc(&drot, sizeof(RotDev)));
        frot.p = drot;
        CUDA_OK(cudaMemcpyAsync(drot, &rd, sizeof(RotDev), cudaMemcpyHostToDevice, s));
        size_t offD, total;
        rotate_offsets(p, n_ct, &offD, &total);
        const size_t ctw = 2ull * p->L * p->N;
        StageLayer sl;
        std::memset(&sl.dev, 0, sizeof(sl.dev));
        LayerDev& L = sl.dev;
        L.in = d_in, L.out = d_out;
        L.R = (u64*)d_ws, L.D = (u64*)((char*)d_ws + offD);
        L.isrc = L.R + ctw, L.isrc_stride = 2 * ctw;  // the rotated copy of every ciphertext
        L.ksk = dkey, L.rots = drot;
        L.n_ct_in = (u32)n_ct, L.n_ct_out = (u32)n_ct, L.n_rot = 2, L.rot_id = 0, L.n_ks = 1;
        L.r_slots = 2, L.r_id = 0;
        run_layers(p, kp, {sl}, s, false, /*do_mac=*/false);
        CUDA_OK(cudaStreamSynchronize(s));
    });
}

// ================================================================== profiling
extern "C" int he_profile_enable(int on) {
    return guard([&] {
        std::lock_guard<std::mutex> lk(g_prof.mu);
        g_prof.on = on != 0;
    });
}
extern "C" int he_profile_collect(he_stage_times* out) {
    return guard([&] {
        if (!out) fail(HE_EINVAL, "null argument");
        std::memset(out, 0, sizeof(*out));
        std::lock_guard<std::mutex> lk(g_prof.mu);
        for (auto& r : g_prof.recs) {
            CUDA_OK(cudaEventSynchronize(r.b));
            float ms = 0;
            CUDA_OK(cudaEventElapsedTime(&ms, r.a, r.b));
            out->ms[r.stage] += ms;
            out->launches[r.stage] += 1;
            g_prof.pool.push_back(r.a);
            g_prof.pool.push_back(r.b);
        }
        g_prof.recs.clear();
    });
}
