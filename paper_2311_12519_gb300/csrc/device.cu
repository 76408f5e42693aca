// Device side of the library (sm_103a): the kernels of one homomorphic
// convolution layer and the plan / forward entry points of the C ABI.
//
// Pipeline of he_conv_forward (Sec. 2.3 hoisting, Sec. 3.1, Sec. 3.2.2):
//   1. k_ntt_inputs   NTT of c0, c1 and of the base-2^w digits of c1 of every
//                     input ciphertext (the "decompose once" half of hoisting)
//   2. k_keyswitch    per rotation: NTT-domain automorphism (an index
//                     permutation) of c0 and the digits, key inner product
//                     with one 128-bit lazy sum and one reduction
//   3. k_mac          lazy CMult/HAdd over input channels, taps and diagonals
//                     with 64-bit split accumulators; one reduction per sum;
//                     epilogue k*A0 + A1 * NTT(P_k) (the [k,-k] PMult)
//   4. k_intt         inverse NTT to coefficient form
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>

#include "internal.h"

using namespace hy;

namespace {

// ------------------------------------------------------------------ constants
struct LimbC {
    u64 q, mu;     // Barrett constant for x < 2^(s+63)
    u32 sm1, pad;  // s - 1
    u64 ninv, ninv_sh;
};
struct KP {
    u32 N, logN, L, l, w;
    LimbC limb[HE_MAX_LIMBS];
    const u64* tw;
    const u64* tw_sh;
    const u64* itw;
    const u64* itw_sh;
};
struct RotDev {
    u32 galois, rot, key, pad;
};

#define CUDA_OK(x)                                                                         \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
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
__device__ __forceinline__ u64 shoup(u64 a, u64 w, u64 wsh, u64 q) {
    u64 qt = __umul64hi(a, wsh);
    u64 r = a * w - qt * q;
    return r >= q ? r - q : r;
}
__device__ __forceinline__ u64 addq(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 subq(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// ------------------------------------------------------------------ NTT in shared memory
// Forward: Cooley-Tukey, natural -> bit-reversed, twiddle psi^rev(m+i) for group i of stage m.
__device__ void ntt_fwd_smem(u64* a, u32 N, u32 logN, const u64* tw, const u64* tw_sh, u64 q) {
    for (u32 m = 1, logt = logN - 1; m < N; m <<= 1, logt--) {
        const u32 t = 1u << logt;
        for (u32 b = threadIdx.x; b < N / 2; b += blockDim.x) {
            u32 i = b >> logt, j = b & (t - 1);
            u32 i1 = (i << (logt + 1)) + j, i2 = i1 + t;
            u64 U = a[i1], V = shoup(a[i2], __ldg(tw + m + i), __ldg(tw_sh + m + i), q);
            a[i1] = addq(U, V, q);
            a[i2] = subq(U, V, q);
        }
        __syncthreads();
    }
}
// Inverse: Gentleman-Sande, bit-reversed -> natural, twiddle psi^-rev(h+i); no 1/N scaling.
__device__ void ntt_inv_smem(u64* a, u32 N, u32 logN, const u64* itw, const u64* itw_sh, u64 q) {
    for (u32 h = N / 2, logt = 0; h >= 1; h >>= 1, logt++) {
        const u32 t = 1u << logt;
        for (u32 b = threadIdx.x; b < N / 2; b += blockDim.x) {
            u32 i = b >> logt, j = b & (t - 1);
            u32 i1 = (i << (logt + 1)) + j, i2 = i1 + t;
            u64 U = a[i1], V = a[i2];
            a[i1] = addq(U, V, q);
            a[i2] = shoup(subq(U, V, q), __ldg(itw + h + i), __ldg(itw_sh + h + i), q);
        }
        __syncthreads();
    }
}

// Step 1: forward NTT of the inputs.  blockIdx.x = ciphertext c; blockIdx.y =
// job: y < 2L -> polynomial y/L, limb y%L into R[c][rot_id]; otherwise digit
// dd = (y-2L)/L of c1 lifted into limb (y-2L)%L, into D[c][dd].
__global__ void k_ntt_inputs(const u64* __restrict__ in, u64* __restrict__ R, u64* __restrict__ D, KP kp,
                             u32 n_rot, u32 rot_id) {
    extern __shared__ u64 sm[];
    const u32 N = kp.N, L = kp.L, l = kp.l;
    const u32 c = blockIdx.x, y = blockIdx.y;
    const size_t ctw = 2ull * L * N;
    const u64* src;
    u64* dst;
    u32 limb, shift = 0;
    bool digit = false;
    if (y < 2 * L) {
        limb = y % L;
        src = in + c * ctw + (size_t)y * N;
        dst = R + ((size_t)c * n_rot + rot_id) * ctw + (size_t)y * N;
    } else {
        u32 z = y - 2 * L, dd = z / L;
        limb = z % L;
        src = in + c * ctw + (size_t)(L + dd / l) * N;
        dst = D + (((size_t)c * L * l + dd) * L + limb) * N;
        shift = kp.w * (dd % l);
        digit = true;
    }
    const LimbC m = kp.limb[limb];
    const u64 mask = (kp.w >= 64) ? ~0ull : ((1ull << kp.w) - 1);
    for (u32 x = threadIdx.x; x < N; x += blockDim.x) {
        u64 v = src[x];
        if (digit) {
            v = (shift >= 64) ? 0 : ((v >> shift) & mask);
            v = v >= m.q ? v - m.q : v;
        }
        sm[x] = v;
    }
    __syncthreads();
    ntt_fwd_smem(sm, N, kp.logN, kp.tw + (size_t)limb * N, kp.tw_sh + (size_t)limb * N, m.q);
    for (u32 x = threadIdx.x; x < N; x += blockDim.x) dst[x] = sm[x];
}

// Plain batched NTT: polynomial blockIdx.x of [n][N], limb = index % L.
__global__ void k_ntt_plain(u64* __restrict__ a, KP kp, int inverse) {
    extern __shared__ u64 sm[];
    const u32 N = kp.N, limb = blockIdx.x % kp.L;
    u64* poly = a + (size_t)blockIdx.x * N;
    const LimbC m = kp.limb[limb];
    for (u32 x = threadIdx.x; x < N; x += blockDim.x) sm[x] = poly[x];
    __syncthreads();
    if (!inverse) {
        ntt_fwd_smem(sm, N, kp.logN, kp.tw + (size_t)limb * N, kp.tw_sh + (size_t)limb * N, m.q);
        for (u32 x = threadIdx.x; x < N; x += blockDim.x) poly[x] = sm[x];
    } else {
        ntt_inv_smem(sm, N, kp.logN, kp.itw + (size_t)limb * N, kp.itw_sh + (size_t)limb * N, m.q);
        for (u32 x = threadIdx.x; x < N; x += blockDim.x) poly[x] = shoup(sm[x], m.ninv, m.ninv_sh, m.q);
    }
}

// Step 4: inverse NTT of ciphertexts.  blockIdx.x = ciphertext, blockIdx.y = polynomial*L + limb.
__global__ void k_intt(const u64* __restrict__ src, size_t src_ct_stride, u64* __restrict__ dst,
                       size_t dst_ct_stride, KP kp) {
    extern __shared__ u64 sm[];
    const u32 N = kp.N, limb = blockIdx.y % kp.L;
    const u64* s = src + blockIdx.x * src_ct_stride + (size_t)blockIdx.y * N;
    u64* d = dst + blockIdx.x * dst_ct_stride + (size_t)blockIdx.y * N;
    const LimbC m = kp.limb[limb];
    for (u32 x = threadIdx.x; x < N; x += blockDim.x) sm[x] = s[x];
    __syncthreads();
    ntt_inv_smem(sm, N, kp.logN, kp.itw + (size_t)limb * N, kp.itw_sh + (size_t)limb * N, m.q);
    for (u32 x = threadIdx.x; x < N; x += blockDim.x) d[x] = shoup(sm[x], m.ninv, m.ninv_sh, m.q);
}

// Step 2: hoisted key switch.  Thread = NTT slot x of limb blockIdx.y;
// blockIdx.z = rotation.  The NTT slot x holds the evaluation at psi^e with
// e = 2 rev(x) + 1, so sigma_g reads slot rev((g e mod 2N - 1)/2).
// The key values of (x, limb) stay in registers across all input ciphertexts.
template <int LL>
__global__ void k_keyswitch(const u64* __restrict__ D, u64* __restrict__ R, const u64* __restrict__ ksk,
                            const RotDev* __restrict__ rots, u32 n_ct, u32 n_rot, u32 rot_id, KP kp) {
    const u32 N = kp.N, L = kp.L, logN = kp.logN;
    const u32 x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const u32 k = blockIdx.y;
    const RotDev rd = rots[blockIdx.z];
    const LimbC m = kp.limb[k];
    const u32 e = 2 * (__brev(x) >> (32 - logN)) + 1;
    const u32 e2 = (u32)(((u64)e * rd.galois) & (2ull * N - 1));
    const u32 src = __brev((e2 - 1) >> 1) >> (32 - logN);
    u64 k0[LL], k1[LL];
    const u64* kb = ksk + (size_t)rd.key * LL * 2 * L * N;
#pragma unroll
    for (int dd = 0; dd < LL; dd++) {
        k0[dd] = kb[(((size_t)dd * 2 + 0) * L + k) * N + x];
        k1[dd] = kb[(((size_t)dd * 2 + 1) * L + k) * N + x];
    }
    const size_t ctw = 2ull * L * N;
    for (u32 c = 0; c < n_ct; c++) {
        const u64* Dc = D + (size_t)c * LL * L * N + (size_t)k * N + src;
        u128 a0 = 0, a1 = 0;
#pragma unroll
        for (int dd = 0; dd < LL; dd++) {
            u64 dv = Dc[(size_t)dd * L * N];
            a0 += (u128)dv * k0[dd];
            a1 += (u128)dv * k1[dd];
        }
        u64* Rc = R + (size_t)c * n_rot * ctw;
        a0 += Rc[(size_t)rot_id * ctw + (size_t)k * N + src];
        Rc[(size_t)rd.rot * ctw + (size_t)k * N + x] = bred128(a0, m);
        Rc[(size_t)rd.rot * ctw + (size_t)(L + k) * N + x] = bred128(a1, m);
    }
}

// Step 3: lazy channel multiply-accumulate (CMult^- and HAdd^128 of Sec. 3.2.2).
// Each residue v < 2^50 is split v = vh 2^25 + vl; s*vl and s*vh accumulate
// exactly in int64 (|s| <= 2^15, at most 2^14 terms), and A = hi 2^25 + lo is
// reduced once.  PACKED: rows r = 0, 1 of the Walsh-Hadamard pair and the
// epilogue out = k*[A0] + [A1] * NTT(P_k); otherwise out = [A0].
constexpr int MAC_THREADS = 256;
constexpr int MAC_KC = 256;

__device__ __forceinline__ u64 reduce_split(i64 lo, i64 hi, const LimbC& m) {
    i128 a = ((i128)hi << 25) + (i128)lo + ((i128)m.q << 32);
    return bred128((u128)a, m);
}

template <int GT, bool PACKED, bool DW>
__global__ void __launch_bounds__(MAC_THREADS) k_mac(const u64* __restrict__ R, u64* __restrict__ OUTN,
                                                     const int16_t* __restrict__ scal, const u64* __restrict__ pk,
                                                     KP kp, u32 in_groups, u32 out_groups, u32 n_rot, u32 K,
                                                     u64 kmul) {
    constexpr int NR = PACKED ? 2 : 1;
    __shared__ int16_t ss[GT][NR][MAC_KC];
    const u32 N = kp.N, L = kp.L;
    const u32 x = blockIdx.x * MAC_THREADS + threadIdx.x;
    const u32 g0 = blockIdx.y * GT;
    const u32 z = blockIdx.z, k = z % L, p = (z / L) & 1, ru = z / (2 * L);
    const LimbC m = kp.limb[k];
    const size_t ctw = 2ull * L * N;
    i64 lo[GT][NR], hi[GT][NR];
#pragma unroll
    for (int g = 0; g < GT; g++)
#pragma unroll
        for (int r = 0; r < NR; r++) lo[g][r] = hi[g][r] = 0;

    for (u32 kc0 = 0; kc0 < K; kc0 += MAC_KC) {
        const u32 kcn = min((u32)MAC_KC, K - kc0);
        for (u32 idx = threadIdx.x; idx < (u32)(GT * NR * MAC_KC); idx += MAC_THREADS) {
            u32 g = idx / (NR * MAC_KC), r = (idx / MAC_KC) % NR, kk = idx % MAC_KC;
            int16_t v = 0;
            if (kk < kcn && g0 + g < out_groups) v = scal[((size_t)(g0 + g) * NR + r) * K + kc0 + kk];
            ss[g][r][kk] = v;
        }
        __syncthreads();
        if (x < N) {
            for (u32 kk = 0; kk < kcn; kk++) {
                const u32 kg = kc0 + kk;
                u32 ct, rot;
                if (DW) {
                    ct = ru * in_groups + g0;
                    rot = kg;
                } else {
                    ct = ru * in_groups + kg / n_rot;
                    rot = kg % n_rot;
                }
                const u64 v = R[((size_t)ct * n_rot + rot) * ctw + ((size_t)p * L + k) * N + x];
                const int vl = (int)(v & 0x1FFFFFFull), vh = (int)(v >> 25);
#pragma unroll
                for (int g = 0; g < GT; g++)
#pragma unroll
                    for (int r = 0; r < NR; r++) {
                        const int s = ss[g][r][kk];
                        lo[g][r] += (i64)s * vl;
                        hi[g][r] += (i64)s * vh;
                    }
            }
        }
        __syncthreads();
    }
    if (x >= N) return;
    const u64 pkv = PACKED ? pk[(size_t)k * N + x] : 0;
#pragma unroll
    for (int g = 0; g < GT; g++) {
        if (g0 + g >= out_groups) break;
        u64 out = reduce_split(lo[g][0], hi[g][0], m);
        if (PACKED) {
            u64 a1 = reduce_split(lo[g][1], hi[g][1], m);
            out = addq(mulmod(kmul, out, m), mulmod(a1, pkv, m), m.q);
        }
        OUTN[((size_t)(ru * out_groups + g0 + g) * 2 + p) * L * N + (size_t)k * N + x] = out;
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
    for (u32 k = 0; k < p->L; k++) {
        kp.limb[k].q = p->q[k];
        kp.limb[k].mu = p->mod[k].mu;
        kp.limb[k].sm1 = p->mod[k].sm1;
        kp.limb[k].ninv = p->ntt[k].ninv;
        kp.limb[k].ninv_sh = p->ntt[k].ninv_sh;
    }
    kp.tw = T.tw, kp.tw_sh = T.tw_sh, kp.itw = T.itw, kp.itw_sh = T.itw_sh;
    return kp;
}

u32 ntt_threads(u32 N) { return std::min<u32>(512, N / 2); }

template <class K>
void allow_smem(K kernel, size_t bytes) {
    CUDA_OK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

void launch_ntt_plain(const he_params* p, const KP& kp, u64* d, int n, int inverse, cudaStream_t s) {
    if (n <= 0) return;
    size_t smem = (size_t)p->N * 8;
    allow_smem(k_ntt_plain, smem);
    k_ntt_plain<<<n, ntt_threads(p->N), smem, s>>>(d, kp, inverse);
    check_launch("k_ntt_plain");
}

template <int LL>
void launch_ks_ll(dim3 grid, cudaStream_t s, const u64* D, u64* R, const u64* ksk, const RotDev* rots, u32 n_ct,
                  u32 n_rot, u32 rot_id, const KP& kp) {
    k_keyswitch<LL><<<grid, 256, 0, s>>>(D, R, ksk, rots, n_ct, n_rot, rot_id, kp);
}

void launch_keyswitch(const he_params* p, const KP& kp, const u64* D, u64* R, const u64* ksk, const RotDev* rots,
                      u32 n_rots, u32 n_ct, u32 n_rot, u32 rot_id, cudaStream_t s) {
    if (!n_rots || !n_ct) return;
    dim3 grid((p->N + 255) / 256, p->L, n_rots);
    const u32 LL = p->L * p->l;
    switch (LL) {
#define KS_CASE(v) \
    case v: launch_ks_ll<v>(grid, s, D, R, ksk, rots, n_ct, n_rot, rot_id, kp); break;
        KS_CASE(1) KS_CASE(2) KS_CASE(3) KS_CASE(4) KS_CASE(5) KS_CASE(6) KS_CASE(7) KS_CASE(8) KS_CASE(9)
            KS_CASE(10) KS_CASE(12) KS_CASE(14) KS_CASE(15) KS_CASE(16)
#undef KS_CASE
        default:
            fail(HE_EINVAL, "L * l must be at most 16 (and not 11 or 13)");
    }
    check_launch("k_keyswitch");
}

void launch_ntt_inputs(const he_params* p, const KP& kp, const u64* in, u64* R, u64* D, u32 n_ct, u32 n_rot,
                       u32 rot_id, cudaStream_t s) {
    if (!n_ct) return;
    size_t smem = (size_t)p->N * 8;
    allow_smem(k_ntt_inputs, smem);
    dim3 grid(n_ct, 2 * p->L + p->L * p->l * p->L);
    k_ntt_inputs<<<grid, ntt_threads(p->N), smem, s>>>(in, R, D, kp, n_rot, rot_id);
    check_launch("k_ntt_inputs");
}

void launch_intt(const he_params* p, const KP& kp, const u64* src, size_t src_stride, u64* dst, size_t dst_stride,
                 u32 n_ct, cudaStream_t s) {
    if (!n_ct) return;
    size_t smem = (size_t)p->N * 8;
    allow_smem(k_intt, smem);
    dim3 grid(n_ct, 2 * p->L);
    k_intt<<<grid, ntt_threads(p->N), smem, s>>>(src, src_stride, dst, dst_stride, kp);
    check_launch("k_intt");
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
    std::vector<u64> tw(n), tws(n), itw(n), itws(n);
    for (u32 k = 0; k < p->L; k++) {
        std::copy(p->ntt[k].tw.begin(), p->ntt[k].tw.end(), tw.begin() + (size_t)k * p->N);
        std::copy(p->ntt[k].tw_sh.begin(), p->ntt[k].tw_sh.end(), tws.begin() + (size_t)k * p->N);
        std::copy(p->ntt[k].itw.begin(), p->ntt[k].itw.end(), itw.begin() + (size_t)k * p->N);
        std::copy(p->ntt[k].itw_sh.begin(), p->ntt[k].itw_sh.end(), itws.begin() + (size_t)k * p->N);
    }
    u64** dst[4] = {&T->tw, &T->tw_sh, &T->itw, &T->itw_sh};
    std::vector<u64>* srcs[4] = {&tw, &tws, &itw, &itws};
    for (int i = 0; i < 4; i++) {
        CUDA_OK(cudaMalloc(dst[i], n * 8));
        CUDA_OK(cudaMemcpy(*dst[i], srcs[i]->data(), n * 8, cudaMemcpyHostToDevice));
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
            cudaFree(t->tw_sh);
            cudaFree(t->itw);
            cudaFree(t->itw_sh);
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
    bool packed = false, dw = false;
    u32 mac_groups = 8;
    u64* d_ksk = nullptr;
    RotDev* d_rots = nullptr;
    int16_t* d_scal = nullptr;
    u64* d_pk = nullptr;
    size_t off_R = 0, off_D = 0, off_O = 0, ws_bytes = 0;
    KP kp{};
    ~he_plan() {
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) return;
        cudaSetDevice(device);
        cudaFree(d_ksk);
        cudaFree(d_rots);
        cudaFree(d_scal);
        cudaFree(d_pk);
        cudaSetDevice(cur);
    }
};

extern "C" int he_conv_plan(const he_params* p, const he_galkeys* gk, const he_conv_desc* d, const int32_t* weights,
                            const he_tune* tune, he_plan** out) {
    return guard([&] {
        if (!p || !gk || !d || !weights || !out) fail(HE_EINVAL, "null argument");
        if (gk->p != p) fail(HE_EINVAL, "Galois keys belong to other parameters");
        *out = nullptr;
        auto P = std::make_unique<he_plan>();
        P->p = p;
        P->d = *d;
        compute_layout(p, d, &P->lay);
        const he_layout& lay = P->lay;
        P->packed = d->c_n == 2;
        P->dw = d->depthwise != 0;
        std::vector<RotEntry> rl = rotation_list(p, d, lay);
        P->n_rot = (u32)rl.size();
        const u32 ndiag = (P->packed && !P->dw) ? 2 : 1;
        const u32 taps = d->kh * d->kh;
        // rotations that need a key switch, grouped by distinct Galois element
        std::vector<u32> gal;
        std::vector<RotDev> rots;
        bool have_id = false;
        for (u32 r = 0; r < rl.size(); r++) {
            if (rl[r].galois == 1) {
                P->rot_id = r;
                have_id = true;
                continue;
            }
            auto it = std::find(gal.begin(), gal.end(), rl[r].galois);
            u32 key = (u32)(it - gal.begin());
            if (it == gal.end()) gal.push_back(rl[r].galois);
            rots.push_back({rl[r].galois, r, key, 0});
        }
        if (!have_id) fail(HE_EINVAL, "internal: identity rotation missing");
        std::vector<const std::vector<u64>*> keys;
        for (u32 g : gal) {
            const std::vector<u64>* k = gk->find(g);
            if (!k) fail(HE_EMISSINGKEY, "missing Galois key " + std::to_string(g));
            keys.push_back(k);
        }
        if (p->L * p->l > 16) fail(HE_EINVAL, "L * l must be at most 16");
        // Hadamard scalars s0 = v0 + v1, s1 = v0 - v1 (Eq. 1 without the 1/2)
        const u32 NR = P->packed ? 2 : 1;
        P->K = P->dw ? P->n_rot : lay.in_groups * P->n_rot;
        if (P->K > (1u << 14)) fail(HE_EINVAL, "too many accumulation terms (C_in kh^2 > 16384)");
        std::vector<int16_t> sc((size_t)lay.out_groups * NR * P->K, 0);
        const u32 wcin = P->dw ? 1 : d->C_in;
        auto W = [&](u32 o, u32 i, u32 tap) -> i64 {
            if (o >= d->C_out || i >= d->C_in) return 0;
            if (P->dw) return o == i ? weights[((size_t)o * 1 + 0) * taps + tap] : 0;
            return weights[((size_t)o * wcin + i) * taps + tap];
        };
        double worst0 = 0, worst1 = 0, worst_abs = 0;
        for (u32 g = 0; g < lay.out_groups; g++) {
            double s0q = 0, s1q = 0, sab = 0;
            for (u32 kk = 0; kk < P->K; kk++) {
                u32 j = P->dw ? g : kk / P->n_rot, r = kk % P->n_rot;
                u32 tap = rl[r].tap, dg = rl[r].d;
                i64 s0, s1 = 0;
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
        }
        (void)ndiag;
        double est = estimate_noise_log2(p, p->w, worst0, worst1, worst_abs, P->packed);
        if (est >= p->log2_delta - 1.0) fail(HE_ENOISE, "estimated noise exceeds Delta/2 for this layer");
        // device data
        CUDA_OK(cudaGetDevice(&P->device));
        P->kp = make_kp(p);
        cudaStream_t s = 0;
        P->d_ksk = upload_keys(p, P->kp, keys, s);
        P->n_ks = (u32)rots.size();
        if (!rots.empty()) {
            CUDA_OK(cudaMalloc(&P->d_rots, rots.size() * sizeof(RotDev)));
            CUDA_OK(cudaMemcpy(P->d_rots, rots.data(), rots.size() * sizeof(RotDev), cudaMemcpyHostToDevice));
        }
        CUDA_OK(cudaMalloc(&P->d_scal, sc.size() * sizeof(int16_t)));
        CUDA_OK(cudaMemcpy(P->d_scal, sc.data(), sc.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
        // NTT(P_k): P_k = kh (X^(N/4) + X^(3N/4)) lifted into every limb
        if (P->packed) {
            std::vector<u64> pk((size_t)p->L * p->N, 0);
            for (u32 k = 0; k < p->L; k++) {
                u64 v = p->mod[k].from_signed(p->kh);
                pk[(size_t)k * p->N + p->N / 4] = v;
                pk[(size_t)k * p->N + 3 * p->N / 4] = v;
                p->ntt[k].forward(pk.data() + (size_t)k * p->N);
            }
            CUDA_OK(cudaMalloc(&P->d_pk, pk.size() * 8));
            CUDA_OK(cudaMemcpy(P->d_pk, pk.data(), pk.size() * 8, cudaMemcpyHostToDevice));
        }
        CUDA_OK(cudaStreamSynchronize(s));
        if (tune && tune->mac_groups) P->mac_groups = tune->mac_groups;
        if (P->dw) P->mac_groups = 1;
        // workspace: R [n_ct_in][n_rot][2][L][N], D [n_ct_in][L l][L][N], O [n_ct_out][2][L][N]
        const size_t ctw = 2ull * p->L * p->N;
        P->off_R = 0;
        P->off_D = align256(P->off_R + (size_t)lay.n_ct_in * P->n_rot * ctw * 8);
        P->off_O = align256(P->off_D + (size_t)lay.n_ct_in * p->L * p->l * p->L * p->N * 8);
        P->ws_bytes = align256(P->off_O + (size_t)lay.n_ct_out * ctw * 8);
        *out = P.release();
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

template <int GT, bool PACKED, bool DW>
static void launch_mac_t(const he_plan* P, const u64* R, u64* O, cudaStream_t s) {
    const he_params* p = P->p;
    dim3 grid((p->N + MAC_THREADS - 1) / MAC_THREADS, (P->lay.out_groups + GT - 1) / GT, P->lay.row_units * 2 * p->L);
    k_mac<GT, PACKED, DW><<<grid, MAC_THREADS, 0, s>>>(R, O, P->d_scal, P->d_pk, P->kp, P->lay.in_groups,
                                                        P->lay.out_groups, P->n_rot, P->K, P->p->k);
}

static void launch_mac(const he_plan* P, const u64* R, u64* O, cudaStream_t s) {
    if (P->dw) {
        if (P->packed) launch_mac_t<1, true, true>(P, R, O, s);
        else launch_mac_t<1, false, true>(P, R, O, s);
    } else if (P->packed) {
        switch (P->mac_groups) {
            case 1: launch_mac_t<1, true, false>(P, R, O, s); break;
            case 2: launch_mac_t<2, true, false>(P, R, O, s); break;
            case 4: launch_mac_t<4, true, false>(P, R, O, s); break;
            default: launch_mac_t<8, true, false>(P, R, O, s); break;
        }
    } else {
        switch (P->mac_groups) {
            case 1: launch_mac_t<1, false, false>(P, R, O, s); break;
            case 2: launch_mac_t<2, false, false>(P, R, O, s); break;
            case 4: launch_mac_t<4, false, false>(P, R, O, s); break;
            case 8: launch_mac_t<8, false, false>(P, R, O, s); break;
            default: launch_mac_t<16, false, false>(P, R, O, s); break;
        }
    }
    check_launch("k_mac");
}

static void forward_impl(const he_plan* P, const u64* d_in, u64* d_out, void* ws, cudaStream_t s, bool timed = true) {
    const he_params* p = P->p;
    if (((uintptr_t)d_in | (uintptr_t)d_out | (uintptr_t)ws) & 15) fail(HE_EINVAL, "device pointers must be 16-byte aligned");
    int dev = -1;
    CUDA_OK(cudaGetDevice(&dev));
    if (dev != P->device) fail(HE_EINVAL, "plan was made on another device");
    char* base = (char*)ws;
    u64* R = (u64*)(base + P->off_R);
    u64* D = (u64*)(base + P->off_D);
    u64* O = (u64*)(base + P->off_O);
    const he_layout& lay = P->lay;
    {
        StageTimer t(HE_STAGE_NTT_IN, s, timed);
        launch_ntt_inputs(p, P->kp, d_in, R, D, lay.n_ct_in, P->n_rot, P->rot_id, s);
    }
    {
        StageTimer t(HE_STAGE_KEYSWITCH, s, timed);
        launch_keyswitch(p, P->kp, D, R, P->d_ksk, P->d_rots, P->n_ks, lay.n_ct_in, P->n_rot, P->rot_id, s);
    }
    {
        StageTimer t(HE_STAGE_MAC, s, timed);
        launch_mac(P, R, O, s);
    }
    {
        StageTimer t(HE_STAGE_NTT_OUT, s, timed);
        const size_t ctw = 2ull * p->L * p->N;
        launch_intt(p, P->kp, O, ctw, d_out, ctw, lay.n_ct_out, s);
    }
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

extern "C" void he_plan_destroy(he_plan* plan) { delete plan; }

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
        cudaStream_t s = (cudaStream_t)stream;
        KP kp = make_kp(p);
        u64* dkey = upload_keys(p, kp, {key}, s);
        RotDev rd{galois, 1, 0, 0};
        RotDev* drot = nullptr;
        CUDA_OK(cudaMalloc(&drot, sizeof(RotDev)));
        CUDA_OK(cudaMemcpyAsync(drot, &rd, sizeof(RotDev), cudaMemcpyHostToDevice, s));
        size_t offD, total;
        rotate_offsets(p, n_ct, &offD, &total);
        u64* R = (u64*)d_ws;
        u64* D = (u64*)((char*)d_ws + offD);
        launch_ntt_inputs(p, kp, d_in, R, D, (u32)n_ct, 2, 0, s);
        launch_keyswitch(p, kp, D, R, dkey, drot, 1, (u32)n_ct, 2, 0, s);
        const size_t ctw = 2ull * p->L * p->N;
        launch_intt(p, kp, R + ctw, 2 * ctw, d_out, ctw, (u32)n_ct, s);
        CUDA_OK(cudaStreamSynchronize(s));
        cudaFree(dkey);
        cudaFree(drot);
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
