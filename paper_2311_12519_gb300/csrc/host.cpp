// Host side of the library: parameter selection (Sec. 3.2.1), the client's
// key generation / encryption / decryption (Sec. 2.3), the slot layout of a
// layer (Sec. 2.4, Sec. 3.1) and the noise estimate that picks the key
// switching base.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "internal.h"

namespace hy {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }
[[noreturn]] void fail(int code, const std::string& msg) { throw Error(code, msg); }

// ------------------------------------------------------------------ modulus
static int bitlen(u64 x) { return x ? 64 - __builtin_clzll(x) : 0; }

Modulus Modulus::make(u64 q) {
    Modulus m;
    m.q = q;
    int s = bitlen(q);
    m.sm1 = (u32)(s - 1);
    // floor(2^(s+63) / q) fits in 64 bits because q >= 2^(s-1)
    u128 num = (u128)1 << (s + 63);
    m.mu = (u64)(num / q);
    return m;
}
u64 Modulus::pow(u64 a, u64 e) const {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mul(r, a);
        a = mul(a, a);
        e >>= 1;
    }
    return r;
}

// ------------------------------------------------------------------ host NTT
void HostNtt::init(int n, u64 q, u64 root) {
    N = n;
    logN = bitlen((u64)n) - 1;
    m = Modulus::make(q);
    psi = root;
    tw.resize(N), tw_sh.resize(N), itw.resize(N), itw_sh.resize(N);
    u64 psi_inv = m.inv(root);
    for (int k = 0; k < N; k++) {
        u32 r = bit_reverse((u32)k, logN);
        tw[k] = m.pow(root, r);
        itw[k] = m.pow(psi_inv, r);
        tw_sh[k] = shoup_of(tw[k], q);
        itw_sh[k] = shoup_of(itw[k], q);
    }
    ninv = m.inv((u64)N % q);
    ninv_sh = shoup_of(ninv, q);
}

static inline u64 shoup_mul(u64 a, u64 w, u64 wsh, u64 q) {
    u64 qt = (u64)(((u128)a * wsh) >> 64);
    u64 r = a * w - qt * q;
    return r >= q ? r - q : r;
}

void HostNtt::forward(u64* a) const {
    const u64 q = m.q;
    int t = N;
    for (int mm = 1; mm < N; mm <<= 1) {
        t >>= 1;
        for (int i = 0; i < mm; i++) {
            u64 W = tw[mm + i], Ws = tw_sh[mm + i];
            int j1 = 2 * i * t;
            for (int j = j1; j < j1 + t; j++) {
                u64 U = a[j], V = shoup_mul(a[j + t], W, Ws, q);
                a[j] = U + V >= q ? U + V - q : U + V;
                a[j + t] = U >= V ? U - V : U + q - V;
            }
        }
    }
}
void HostNtt::inverse(u64* a) const {
    const u64 q = m.q;
    int t = 1;
    for (int mm = N; mm > 1; mm >>= 1) {
        int h = mm >> 1, j1 = 0;
        for (int i = 0; i < h; i++) {
            u64 W = itw[h + i], Ws = itw_sh[h + i];
            for (int j = j1; j < j1 + t; j++) {
                u64 U = a[j], V = a[j + t];
                a[j] = U + V >= q ? U + V - q : U + V;
                a[j + t] = shoup_mul(U >= V ? U - V : U + q - V, W, Ws, q);
            }
            j1 += 2 * t;
        }
        t <<= 1;
    }
    for (int j = 0; j < N; j++) a[j] = shoup_mul(a[j], ninv, ninv_sh, q);
}

// ------------------------------------------------------------------ big integers
Big big_mul_u64(const Big& a, u64 b) {
    Big r;
    r.w.resize(a.w.size() + 1);
    u64 carry = 0;
    for (size_t i = 0; i < a.w.size(); i++) {
        u128 p = (u128)a.w[i] * b + carry;
        r.w[i] = (u64)p;
        carry = (u64)(p >> 64);
    }
    r.w[a.w.size()] = carry;
    r.trim();
    return r;
}
Big big_add(const Big& a, const Big& b) {
    Big r;
    size_t n = std::max(a.w.size(), b.w.size());
    r.w.resize(n + 1);
    u64 c = 0;
    for (size_t i = 0; i < n; i++) {
        u128 s = (u128)(i < a.w.size() ? a.w[i] : 0) + (i < b.w.size() ? b.w[i] : 0) + c;
        r.w[i] = (u64)s;
        c = (u64)(s >> 64);
    }
    r.w[n] = c;
    r.trim();
    return r;
}
Big big_sub(const Big& a, const Big& b) {
    Big r;
    r.w.resize(a.w.size());
    u64 borrow = 0;
    for (size_t i = 0; i < a.w.size(); i++) {
        u64 bi = i < b.w.size() ? b.w[i] : 0;
        u128 d = (u128)a.w[i] - bi - borrow;
        r.w[i] = (u64)d;
        borrow = (u64)(d >> 64) ? 1 : 0;
    }
    r.trim();
    return r;
}
int big_cmp(const Big& a, const Big& b) {
    size_t n = std::max(a.w.size(), b.w.size());
    for (size_t i = n; i-- > 0;) {
        u64 x = i < a.w.size() ? a.w[i] : 0, y = i < b.w.size() ? b.w[i] : 0;
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}
u64 big_mod_u64(const Big& a, u64 m) {
    u128 r = 0;
    for (size_t i = a.w.size(); i-- > 0;) r = ((r << 64) | a.w[i]) % m;
    return (u64)r;
}
double big_log2(const Big& a) {
    size_t n = a.w.size();
    double v = (double)a.w[n - 1];
    if (n >= 2) v += (double)a.w[n - 2] / 18446744073709551616.0;
    return std::log2(v) + 64.0 * (double)(n - 1);
}
u64 big_div_small_quotient(const Big& a, const Big& b) {
    // binary long division of the quotient bits, highest first
    u64 qv = 0;
    for (int bit = 63; bit >= 0; bit--) {
        u64 cand = qv | (1ULL << bit);
        if (big_cmp(big_mul_u64(b, cand), a) <= 0) qv = cand;
    }
    return qv;
}

// ------------------------------------------------------------------ primes
static bool miller_rabin(u64 n) {
    if (n < 2) return false;
    static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : small)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) d >>= 1, r++;
    Modulus m = Modulus::make(n);
    for (u64 a : small) {
        u64 x = m.pow(a, d);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; i++) {
            x = m.mul(x, x);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}
// primes p < 2^bits with p = 1 mod 2N, from the top down
static std::vector<u64> primes_below(u32 bits, u64 twoN, u32 count) {
    std::vector<u64> out;
    u64 top = (bits >= 64) ? ~0ULL : ((1ULL << bits) - 1);
    u64 c = (top / twoN) * twoN + 1;
    if (c > top) c -= twoN;
    while (out.size() < count && c > twoN) {
        if (miller_rabin(c)) out.push_back(c);
        c -= twoN;
    }
    if (out.size() < count) fail(HE_EINVAL, "not enough primes = 1 mod 2N below 2^bits");
    return out;
}
// psi = x^((q-1)/2N) for the smallest quadratic non-residue x (then psi^N = -1)
static u64 root_2n(u64 q, u64 N) {
    Modulus m = Modulus::make(q);
    for (u64 x = 2;; x++)
        if (m.pow(x, (q - 1) / 2) == q - 1) return m.pow(x, (q - 1) / (2 * N));
}
// the smallest x with x^N = -1 mod t: it fixes the slot order of the encoding
static u64 min_root_2n(u64 t, u64 N) {
    Modulus m = Modulus::make(t);
    for (u64 x = 2; x < t; x++)
        if (m.pow(x, N) == t - 1) return x;
    fail(HE_EINVAL, "no primitive 2N-th root mod t");
}

// ------------------------------------------------------------------ random streams
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), read at counter positions.
struct SplitMix {
    static u64 out(u64 state) {
        u64 z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    // n-th output of the generator started at state `key`
    static u64 at(u64 key, u64 n) { return out(key + 0x9E3779B97F4A7C15ULL * (n + 1)); }
    static u64 stream(u64 seed, u64 tag, u64 a, u64 b) { return at(at(at(seed, tag), a), b); }
};

// One draw sequence with the exact samplers of Canonne, Kamath and Steinke,
// "The Discrete Gaussian for Differential Privacy" (2020).
class ExactSampler {
   public:
    explicit ExactSampler(u64 key) : key_(key), n_(0) {}
    u64 next() { return SplitMix::at(key_, n_++); }
    // uniform in [0, m): reject draws below 2^64 mod m
    u64 below(u64 m) {
        const u64 reject_under = (0ULL - m) % m;
        for (;;) {
            u64 x = next();
            if (x >= reject_under) return x % m;
        }
    }
    bool bernoulli(u64 num, u64 den) { return below(den) < num; }
    // Algorithm 1: Bernoulli(exp(-num/den))
    bool bernoulli_exp(u64 num, u64 den) {
        if (num <= den) {
            u64 K = 1;
            for (;;) {
                if (!bernoulli(num, den * K)) break;
                ++K;
            }
            return (K % 2) == 1;
        }
        for (u64 i = num / den; i > 0; --i)
            if (!bernoulli_exp(1, 1)) return false;
        return bernoulli_exp(num % den, den);
    }
    // Algorithm 2 with scale t (s = 1)
    i64 laplace(u64 t) {
        for (;;) {
            u64 U = below(t);
            if (!bernoulli_exp(U, t)) continue;
            u64 V = 0;
            while (bernoulli_exp(1, 1)) ++V;
            u64 X = U + t * V;
            bool neg = bernoulli(1, 2);
            if (neg && X == 0) continue;
            return neg ? -(i64)X : (i64)X;
        }
    }
    // Algorithm 3 with sigma^2 = sn/sd, then truncation to |y| <= bound
    i64 gaussian(u64 sn, u64 sd, i64 bound) {
        u64 t = 1;
        while (t * t * sd <= sn) ++t;  // floor(sigma) + 1
        for (;;) {
            i64 Y = laplace(t);
            u64 a = (u64)(Y < 0 ? -Y : Y);
            i64 c = (i64)(a * t * sd) - (i64)sn;  // (|Y| - sigma^2/t) * t sd
            u64 num = (u64)(c < 0 ? -c : c);
            if (!bernoulli_exp(num * num, 2 * t * t * sd * sn)) continue;
            if (Y < -bound || Y > bound) continue;
            return Y;
        }
    }

   private:
    u64 key_, n_;
};

enum : u64 { TAG_SECRET = 1, TAG_ENC_A = 2, TAG_ENC_E = 3, TAG_KSK_A = 4, TAG_KSK_E = 5 };
static const u64 SIGMA2_NUM = 256, SIGMA2_DEN = 25;  // sigma = 3.2
static const i64 NOISE_BOUND = 32;                    // B = 10 sigma

// uniform residues: limb k, coefficient n from draws 2(kN+n) and 2(kN+n)+1 (128 bits mod q_k)
static void sample_uniform_rns(const he_params* p, u64 key, u64* out) {
    for (u32 k = 0; k < p->L; k++)
        for (u32 n = 0; n < p->N; n++) {
            u64 idx = 2 * ((u64)k * p->N + n);
            u128 x = ((u128)SplitMix::at(key, idx) << 64) | SplitMix::at(key, idx + 1);
            out[(size_t)k * p->N + n] = (u64)(x % p->q[k]);
        }
}
static void sample_gauss(const he_params* p, u64 key, i64* out) {
    for (u32 n = 0; n < p->N; n++) {
        ExactSampler smp(SplitMix::at(key, n));
        out[n] = smp.gaussian(SIGMA2_NUM, SIGMA2_DEN, NOISE_BOUND);
    }
}

// ------------------------------------------------------------------ ring helpers
// c = a * b mod (X^N + 1, q_k) with b given by signed small coefficients
// c = a * s in limb k, with the secret's NTT from key generation
static void mul_secret(const he_params* p, const he_seckey* sk, u32 k, const u64* a, u64* c) {
    const HostNtt& T = p->ntt[k];
    const u64* S = sk->s_ntt.data() + (size_t)k * p->N;
    std::vector<u64> A(a, a + p->N);
    T.forward(A.data());
    for (u32 n = 0; n < p->N; n++) c[n] = p->mod[k].mul(A[n], S[n]);
    T.inverse(c);
}
// Runs fn(i) for every i in [0, n) on up to 64 host threads; independent items only.  The
// first exception a worker throws is rethrown here after all workers have stopped.
template <class F>
static void parallel_for(u32 n, F fn) {
    const u32 T = std::min<u32>({n, 64u, std::max(1u, std::thread::hardware_concurrency())});
    if (T <= 1) {
        for (u32 i = 0; i < n; i++) fn(i);
        return;
    }
    std::atomic<u32> next{0};
    std::exception_ptr err;
    std::mutex mu;
    auto work = [&] {
        try {
            for (u32 i = next++; i < n; i = next++) fn(i);
        } catch (...) {
            std::lock_guard<std::mutex> g(mu);
            if (!err) err = std::current_exception();
            next = n;
        }
    };
    std::vector<std::thread> th;
    for (u32 t = 1; t < T; t++) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
    if (err) std::rethrow_exception(err);
}
// sigma_g on signed coefficients: X^i -> X^(i g mod 2N), negated past N
static void automorph_signed(u32 N, u32 g, const i64* a, i64* out) {
    u64 M = 2ULL * N;
    for (u32 i = 0; i < N; i++) {
        u64 j = ((u64)i * g) % M;
        if (j < N) out[j] = a[i];
        else out[j - N] = -a[i];
    }
}

}  // namespace hy

using namespace hy;

// ================================================================== C ABI
extern "C" const char* he_last_error(void) { return g_last_error.c_str(); }

static void finish_params(he_params* P) {
    const u32 N = P->N;
    P->mod.clear();
    P->ntt.assign(P->L, HostNtt());
    for (u32 k = 0; k < P->L; k++) {
        P->mod.push_back(Modulus::make(P->q[k]));
        P->psi.push_back(root_2n(P->q[k], N));
        P->ntt[k].init((int)N, P->q[k], P->psi[k]);
    }
    P->mod_t = Modulus::make(P->t);
    P->zeta = min_root_2n(P->t, N);
    P->ntt_t.init((int)N, P->t, P->zeta);
    // h_{p,n}: [1,-1] = h (X^(N/4) + X^(3N/4)) with h (w + w^3) = 1, w = zeta^(N/4)
    u64 w8 = P->mod_t.pow(P->zeta, N / 4);
    u64 s = P->mod_t.add(w8, P->mod_t.pow(w8, 3));
    P->h = P->mod_t.inv(s);
    // Q, Delta, CRT basis
    Big Q = Big::from_u64(1);
    for (u64 qi : P->q) Q = big_mul_u64(Q, qi);
    P->Q = Q;
    // Delta = floor(Q / t): long division by a 64-bit word
    {
        Big d;
        d.w.assign(Q.w.size(), 0);
        u128 r = 0;
        for (size_t i = Q.w.size(); i-- > 0;) {
            u128 cur = (r << 64) | Q.w[i];
            d.w[i] = (u64)(cur / P->t);
            r = cur % P->t;
        }
        d.trim();
        P->delta = d;
    }
    P->delta_mod.clear();
    P->crt_Qk.clear();
    P->crt_inv.clear();
    for (u32 k = 0; k < P->L; k++) {
        P->delta_mod.push_back(big_mod_u64(P->delta, P->q[k]));
        Big Qk = Big::from_u64(1);
        for (u32 j = 0; j < P->L; j++)
            if (j != k) Qk = big_mul_u64(Qk, P->q[j]);
        P->crt_inv.push_back(P->mod[k].inv(big_mod_u64(Qk, P->q[k])));
        P->crt_Qk.push_back(Qk);
    }
    P->log2_delta = big_log2(P->delta);
    // NTT position of each flat slot: exponent e = (-1)^r 3^i mod 2N -> rev((e-1)/2)
    P->slot_index.resize(N);
    u64 M = 2ULL * N, e = 1;
    for (u32 i = 0; i < N / 2; i++) {
        P->slot_index[i] = bit_reverse((u32)((e - 1) / 2), (int)P->logN);
        u64 e2 = M - e;
        P->slot_index[N / 2 + i] = bit_reverse((u32)((e2 - 1) / 2), (int)P->logN);
        e = (e * 3) % M;
    }
}

static void hadamard4_setup(he_params* P);

extern "C" int he_params_create(const he_param_req* req, he_params** out) {
    return guard([&] {
        if (!req || !out) fail(HE_EINVAL, "null argument");
        *out = nullptr;
        u32 N = req->N;
        if (N < 1024 || N > 16384 || (N & (N - 1))) fail(HE_EINVAL, "N must be a power of two in [1024, 16384]");
        if (req->L < 1 || req->L > HE_MAX_LIMBS) fail(HE_EINVAL, "L out of range");
        u32 lb = req->limb_bits ? req->limb_bits : 50;
        if (lb < 30 || lb > 54) fail(HE_EINVAL, "limb_bits must be in [30, 54]");
        auto P = std::make_unique<he_params>();
        P->N = N;
        P->L = req->L;
        P->logN = (u32)(bitlen(N) - 1);
        u64 twoN = 2ULL * N;
        if (req->t) {
            if (!miller_rabin(req->t) || req->t % twoN != 1) fail(HE_EINVAL, "t must be a prime = 1 mod 2N");
            if (req->t >= (1ULL << 40)) fail(HE_EINVAL, "t must be below 2^40");
            P->t = req->t;
        } else {
            u32 tb = req->t_bits ? req->t_bits : 20;
            if (tb < 12 || tb > 40) fail(HE_EINVAL, "t_bits must be in [12, 40]");
            P->t = primes_below(tb, twoN, 1)[0];
        }
        P->q = primes_below(lb, twoN, P->L);
        finish_params(P.get());
        // k in [1, k_max] minimising |centred(k h mod t)|
        u32 kmax = req->k_max ? req->k_max : 32;
        u64 best_k = 1, best_v = ~0ULL;
        for (u64 k = 1; k <= kmax; k++) {
            u64 v = P->mod_t.mul(k % P->t, P->h);
            u64 a = v > P->t / 2 ? P->t - v : v;
            if (a < best_v) best_v = a, best_k = k;
        }
        P->k = best_k;
        {
            u64 v = P->mod_t.mul(best_k, P->h);
            P->kh = v > P->t / 2 ? (i64)v - (i64)P->t : (i64)v;
        }
        hadamard4_setup(P.get());
        // decomposition base
        u32 sb = 0;
        for (u64 qi : P->q) sb = std::max(sb, (u32)bitlen(qi));
        if (req->decomp_bits) {
            if (req->decomp_bits < 4 || req->decomp_bits > sb) fail(HE_EINVAL, "decomp_bits out of range");
            P->w = req->decomp_bits;
            double K = req->est_mac_terms ? req->est_mac_terms : 0;
            double W = req->est_weight_max ? req->est_weight_max : 8;
            P->est_noise_log2 = estimate_noise_log2(P.get(), P->w, K * 4 * W * W, K * 4 * W * W, K * 2 * W, true);
        } else {
            if (!req->est_mac_terms) fail(HE_EINVAL, "decomp_bits = 0 needs est_mac_terms");
            double K = req->est_mac_terms;
            double W = req->est_weight_max ? req->est_weight_max : 8;
            bool found = false;
            for (u32 digits = 1; digits <= sb; digits++) {
                u32 w = (sb + digits - 1) / digits;
                double est = estimate_noise_log2(P.get(), w, K * 4 * W * W, K * 4 * W * W, K * 2 * W, true);
                if (est < P->log2_delta - 2.0) {
                    P->w = w;
                    P->est_noise_log2 = est;
                    found = true;
                    break;
                }
            }
            if (!found) fail(HE_ENOISE, "no decomposition base keeps the noise below Delta/4");
        }
        P->l = (sb + P->w - 1) / P->w;
        *out = P.release();
    });
}

extern "C" int he_params_info(const he_params* p, he_param_info* o) {
    return guard([&] {
        if (!p || !o) fail(HE_EINVAL, "null argument");
        std::memset(o, 0, sizeof(*o));
        o->N = p->N, o->L = p->L, o->w = p->w, o->l = p->l;
        o->t = p->t, o->zeta = p->zeta, o->h = p->h, o->k = p->k, o->kh = p->kh, o->k4 = p->k4;
        o->log2_delta = p->log2_delta;
        o->est_noise_log2 = p->est_noise_log2;
        for (u32 k = 0; k < p->L; k++) o->q[k] = p->q[k];
    });
}

extern "C" void he_params_destroy(he_params* p) { delete p; }

// ------------------------------------------------------------------ noise estimate
namespace hy {
// variance of a rotated copy's noise: the key switch sums L*l digit polynomials times sigma(d) * e,
// N terms per coefficient, plus the input's own noise
static double key_switch_variance(const he_params* p, u32 w) {
    u32 sb = 0;
    for (u64 qi : p->q) sb = std::max(sb, (u32)bitlen(qi));
    double l = (double)((sb + w - 1) / w);
    double sigma2 = (double)SIGMA2_NUM / (double)SIGMA2_DEN;
    double d2 = std::ldexp(1.0, (int)(2 * w)) / 3.0;  // E[d^2], d uniform in [0, 2^w)
    return (double)p->L * l * (double)p->N * d2 * sigma2 + sigma2;
}

double estimate_noise_log2(const he_params* p, u32 w, double sum_s0_sq, double sum_s1_sq, double sum_abs_s,
                           bool packed) {
    double var_ks = key_switch_variance(p, w);
    double k = (double)p->k, kh = (double)std::llabs(p->kh), t = (double)p->t;
    double var_out, extra;
    if (packed) {
        var_out = k * k * var_ks * sum_s0_sq + 2.0 * kh * kh * var_ks * sum_s1_sq;
        extra = t * (k * sum_abs_s + 2.0 * kh * sum_abs_s + 2.0 * kh);
    } else {
        var_out = var_ks * sum_s0_sq;
        extra = t * sum_abs_s;
    }
    return std::log2(6.0 * std::sqrt(var_out) + extra + 1.0);
}

// PMult by the k4-scaled pattern b multiplies a noise coefficient by each of its (one or two)
// non-zero coefficients: variance x their sum of squares, worst case x their absolute sum
double estimate_noise_log2_h4(const he_params* p, u32 w, const double sum_sq[4], double sum_abs_s) {
    const double var_ks = key_switch_variance(p, w), k = (double)p->k4, t = (double)p->t;
    double var_out = k * k * var_ks * sum_sq[0], l1 = 0;
    for (u32 b = 0; b < 3; b++) {
        double l2 = 0;
        for (u32 j = 0; j < p->N; j++) {
            const i64 a = p->pat4[(size_t)b * p->N + j];
            if (!a) continue;
            i64 v = (i64)(((__int128)a * (i64)p->k4) % (i64)p->t);
            if (v > (i64)(p->t / 2)) v -= (i64)p->t;
            if (v < -(i64)(p->t / 2)) v += (i64)p->t;
            l2 += (double)v * (double)v, l1 += std::fabs((double)v);
        }
        var_out += l2 * var_ks * sum_sq[b + 1];
    }
    const double extra = t * ((k + l1) * sum_abs_s + l1);
    return std::log2(6.0 * std::sqrt(var_out) + extra + 1.0);
}
}  // namespace hy

// ------------------------------------------------------------------ keys
extern "C" int he_keygen(const he_params* p, uint64_t seed, he_seckey** out) {
    return guard([&] {
        if (!p || !out) fail(HE_EINVAL, "null argument");
        auto sk = std::make_unique<he_seckey>();
        sk->p = p;
        sk->s.resize(p->N);
        u64 key = SplitMix::stream(seed, TAG_SECRET, 0, 0);
        for (u32 n = 0; n < p->N; n++) sk->s[n] = (i64)(SplitMix::at(key, n) % 3) - 1;
        sk->s_ntt.resize((size_t)p->L * p->N);
        for (u32 k = 0; k < p->L; k++) {
            u64* S = sk->s_ntt.data() + (size_t)k * p->N;
            for (u32 n = 0; n < p->N; n++) S[n] = p->mod[k].from_signed(sk->s[n]);
            p->ntt[k].forward(S);
        }
        *out = sk.release();
    });
}
extern "C" int he_seckey_export(const he_seckey* sk, int64_t* c) {
    return guard([&] {
        if (!sk || !c) fail(HE_EINVAL, "null argument");
        std::memcpy(c, sk->s.data(), sizeof(i64) * sk->s.size());
    });
}
extern "C" void he_seckey_destroy(he_seckey* sk) { delete sk; }

extern "C" int he_galois_keys(const he_params* p, const he_seckey* sk, const uint32_t* galois, int n, uint64_t seed,
                              he_galkeys** out) {
    return guard([&] {
        if (!p || !sk || !out || (n > 0 && !galois)) fail(HE_EINVAL, "null argument");
        if (sk->p != p) fail(HE_EINVAL, "secret key belongs to other parameters");
        const u32 N = p->N, L = p->L, l = p->l;
        auto gk = std::make_unique<he_galkeys>();
        gk->p = p;
        for (int gi = 0; gi < n; gi++) {
            u32 g = galois[gi];
            if ((g & 1) == 0 || g >= 2 * N || g == 1) fail(HE_EINVAL, "Galois element must be odd, in [3, 2N)");
            if (std::find(gk->galois.begin(), gk->galois.end(), g) == gk->galois.end()) gk->galois.push_back(g);
        }
        gk->keys.resize(gk->galois.size());
        // every (element, digit) key is drawn from its own counter stream, so elements are independent
        parallel_for((u32)gk->galois.size(), [&](u32 gi) {
            const u32 g = gk->galois[gi];
            std::vector<i64> sg(N), e(N);
            std::vector<u64> a((size_t)L * N), as(N);
            automorph_signed(N, g, sk->s.data(), sg.data());
            std::vector<u64> key((size_t)L * l * 2 * L * N);
            for (u32 i = 0; i < L; i++)
                for (u32 j = 0; j < l; j++) {
                    u32 dd = i * l + j;
                    sample_uniform_rns(p, SplitMix::stream(seed, TAG_KSK_A, g, dd), a.data());
                    sample_gauss(p, SplitMix::stream(seed, TAG_KSK_E, g, dd), e.data());
                    for (u32 k = 0; k < L; k++) {
                        const Modulus& m = p->mod[k];
                        mul_secret(p, sk, k, a.data() + (size_t)k * N, as.data());
                        u64 gadget = (k == i) ? m.pow(2, (u64)p->w * j) : 0;
                        u64* b_out = key.data() + (((size_t)dd * 2 + 0) * L + k) * N;
                        u64* a_out = key.data() + (((size_t)dd * 2 + 1) * L + k) * N;
                        for (u32 x = 0; x < N; x++) {
                            u64 v = m.sub(m.from_signed(e[x]), as[x]);
                            v = m.add(v, m.mul(gadget, m.from_signed(sg[x])));
                            b_out[x] = v;
                            a_out[x] = a[(size_t)k * N + x];
                        }
                    }
                }
            gk->keys[gi] = std::move(key);
        });
        *out = gk.release();
    });
}
extern "C" int he_galkeys_export(const he_galkeys* gk, uint32_t g, uint64_t* out) {
    return guard([&] {
        if (!gk || !out) fail(HE_EINVAL, "null argument");
        const std::vector<u64>* k = gk->find(g);
        if (!k) fail(HE_EMISSINGKEY, "no key for this Galois element");
        std::memcpy(out, k->data(), sizeof(u64) * k->size());
    });
}
extern "C" void he_galkeys_destroy(he_galkeys* gk) { delete gk; }

// ------------------------------------------------------------------ encrypt / decrypt
static void encode_slots(const he_params* p, const int64_t* slots, std::vector<u64>& m) {
    m.assign(p->N, 0);
    for (u32 s = 0; s < p->N; s++) m[p->slot_index[s]] = p->mod_t.from_signed(slots[s]);
    p->ntt_t.inverse(m.data());
}
static void decode_slots(const he_params* p, std::vector<u64>& m, int64_t* slots) {
    p->ntt_t.forward(m.data());
    for (u32 s = 0; s < p->N; s++) slots[s] = (int64_t)m[p->slot_index[s]];
}

// c_n = 4 (Sec. 3.1's 4 x 4 Walsh-Hadamard basis over the slot classes c = 2 row + (index mod 2)):
// the patterns holding H4[b][c] in the slots of class c, b = 1, 2, 3, as centred coefficients,
// and k4, the k in [1, min(t - 1, 2^20)] minimising k + sum |[k a]_t| over their non-zero
// coefficients a (the noise-growth bound of CMult by k and the three PMults; ties -> smallest k).
static const int H4_BASIS[4][4] = {{1, 1, 1, 1}, {1, -1, 1, -1}, {1, 1, -1, -1}, {1, -1, -1, 1}};
static void hadamard4_setup(he_params* P) {
    const u32 N = P->N, half = N / 2;
    P->pat4.assign(3 * (size_t)N, 0);
    std::vector<int64_t> slots(N);
    std::vector<u64> m, nz;
    for (int b = 1; b < 4; b++) {
        for (u32 s = 0; s < N; s++) slots[s] = H4_BASIS[b][2 * (s / half) + (s & 1)];
        encode_slots(P, slots.data(), m);
        for (u32 j = 0; j < N; j++) {
            P->pat4[(size_t)(b - 1) * N + j] = m[j] > P->t / 2 ? (i64)m[j] - (i64)P->t : (i64)m[j];
            if (m[j]) nz.push_back(m[j]);
        }
    }
    const u64 kmax = std::min<u64>(P->t - 1, 1ull << 20);
    std::vector<u64> ka(nz.size(), 0);  // [k a]_t, stepped by a
    u64 best = ~0ull, best_k = 1;
    for (u64 k = 1; k <= kmax; k++) {
        u64 G = k;
        for (size_t i = 0; i < nz.size(); i++) {
            u64 v = ka[i] + nz[i];
            if (v >= P->t) v -= P->t;
            ka[i] = v;
            G += std::min(v, P->t - v);
        }
        if (G < best) best = G, best_k = k;
    }
    P->k4 = best_k;
}
static void encrypt_poly(const he_params* p, const he_seckey* sk, const std::vector<u64>& m, u64 seed, u64 index,
                         u64* ct) {
    const u32 N = p->N, L = p->L;
    std::vector<u64> a((size_t)L * N), as(N);
    std::vector<i64> e(N);
    sample_uniform_rns(p, SplitMix::stream(seed, TAG_ENC_A, index, 0), a.data());
    sample_gauss(p, SplitMix::stream(seed, TAG_ENC_E, index, 0), e.data());
    for (u32 k = 0; k < L; k++) {
        const Modulus& md = p->mod[k];
        mul_secret(p, sk, k, a.data() + (size_t)k * N, as.data());
        u64* c0 = ct + (size_t)k * N;
        u64* c1 = ct + (size_t)(L + k) * N;
        for (u32 x = 0; x < N; x++) {
            u64 v = md.mul(p->delta_mod[k], m[x]);
            v = md.add(v, as[x]);
            c0[x] = md.add(v, md.from_signed(e[x]));
            c1[x] = md.sub(0, a[(size_t)k * N + x]);
        }
    }
}
// m = round(t [c0 + c1 s]_q / q) mod t, exact with multi-word integers
static void decrypt_poly(const he_params* p, const he_seckey* sk, const u64* ct, std::vector<u64>& m) {
    const u32 N = p->N, L = p->L;
    std::vector<u64> ph((size_t)L * N), cs(N);
    for (u32 k = 0; k < L; k++) {
        mul_secret(p, sk, k, ct + (size_t)(L + k) * N, cs.data());
        for (u32 x = 0; x < N; x++) ph[(size_t)k * N + x] = p->mod[k].add(ct[(size_t)k * N + x], cs[x]);
    }
    m.assign(N, 0);
    Big twoQ = big_mul_u64(p->Q, 2);
    for (u32 x = 0; x < N; x++) {
        Big X = Big::from_u64(0);
        // X = sum_k [x_k (Q/q_k)^-1]_{q_k} (Q/q_k): every term is below Q, the sum below L Q
        for (u32 k = 0; k < L; k++)
            X = big_add(X, big_mul_u64(p->crt_Qk[k], p->mod[k].mul(ph[(size_t)k * N + x], p->crt_inv[k])));
        for (u32 k = 0; k < L && big_cmp(X, p->Q) >= 0; k++) X = big_sub(X, p->Q);
        // X in [0, Q); the centred lift differs by a multiple of Q, which shifts
        // the rounded quotient by a multiple of t, so it can be skipped
        Big num = big_add(big_mul_u64(X, 2 * p->t), p->Q);
        m[x] = big_div_small_quotient(num, twoQ) % p->t;
    }
}

extern "C" int he_encrypt_slots(const he_params* p, const he_seckey* sk, const int64_t* slots, uint64_t seed,
                                uint64_t index, uint64_t* ct) {
    return guard([&] {
        if (!p || !sk || !slots || !ct) fail(HE_EINVAL, "null argument");
        std::vector<u64> m;
        encode_slots(p, slots, m);
        encrypt_poly(p, sk, m, seed, index, ct);
    });
}
extern "C" int he_decrypt_slots(const he_params* p, const he_seckey* sk, const uint64_t* ct, int64_t* slots) {
    return guard([&] {
        if (!p || !sk || !slots || !ct) fail(HE_EINVAL, "null argument");
        std::vector<u64> m;
        decrypt_poly(p, sk, ct, m);
        decode_slots(p, m, slots);
    });
}

// ------------------------------------------------------------------ layout
namespace hy {
static void choose_tile(u32 half, u32 H, u32 W, u32 P, u32 S, u32* Th, u32* Tw) {
    if ((H + 2 * P) * (W + 2 * P) <= half) {
        *Th = H, *Tw = W;
        return;
    }
    if ((W + 2 * P) * (S + 2 * P) <= half) {
        u32 rows = half / (W + 2 * P) - 2 * P;
        *Th = std::min((rows / S) * S, H);
        *Tw = W;
        return;
    }
    u32 tw = S;
    while (tw + S <= W && (tw + S + 2 * P) * (tw + S + 2 * P) <= half) tw += S;
    if ((tw + 2 * P) * (S + 2 * P) > half) fail(HE_EINVAL, "kernel too large for the ring degree");
    u32 rows = half / (tw + 2 * P) - 2 * P;
    *Th = std::min((rows / S) * S, H);
    *Tw = tw;
}

u32 rotation_galois(const he_params* p, i64 step) {
    i64 half = p->N / 2;
    i64 s = ((step % half) + half) % half;
    u64 M = 2ULL * p->N, g = 1, b = 3;
    for (u64 e = (u64)s; e; e >>= 1) {
        if (e & 1) g = g * b % M;
        b = b * b % M;
    }
    return (u32)g;
}

// The plane geometry a layer's slots hold: the image itself, or for polyphase packing the four
// phase planes in[2u + a][2v + b] of ceil(H/2) x ceil(W/2), each a channel of a stride-1 layer.
void plane_geometry(const he_conv_desc* d, u32* H, u32* W, u32* S, u32* C_planes) {
    if (d->polyphase) {
        *H = (d->H + 1) / 2, *W = (d->W + 1) / 2, *S = 1;
        *C_planes = 4 * ((d->C_in + d->c_n - 1) / d->c_n * d->c_n);
    } else {
        *H = d->H, *W = d->W, *S = d->stride, *C_planes = d->C_in;
    }
}

void compute_layout(const he_params* p, const he_conv_desc* d, he_layout* o) {
    if (!d->C_in || !d->C_out || !d->H || !d->W || !d->n_images) fail(HE_EINVAL, "empty layer");
    if (d->kh % 2 == 0 || d->kh > 7) fail(HE_EINVAL, "kernel must be odd, at most 7");
    if (d->stride < 1 || d->stride > 2) fail(HE_EINVAL, "stride must be 1 or 2");
    if (d->c_n != 1 && d->c_n != 2 && d->c_n != 4) fail(HE_EINVAL, "c_n must be 1, 2 or 4");
    if (d->depthwise && d->C_in != d->C_out) fail(HE_EINVAL, "depthwise needs C_in == C_out");
    if (d->polyphase > 1 || (d->polyphase && (d->stride != 2 || d->kh != 3)))
        fail(HE_EINVAL, "polyphase packing is for 3x3 stride-2 layers (polyphase 0 or 1)");
    if (d->c_n == 4 && d->polyphase) fail(HE_EINVAL, "polyphase packing is built for c_n 1 and 2");
    std::memset(o, 0, sizeof(*o));
    // block positions of a slot row: N/2, or N/4 with c_n = 4 (two slot parities per position)
    const u32 half = d->c_n == 4 ? p->N / 4 : p->N / 2, P = (d->kh - 1) / 2;
    u32 Hp, Wp, S, Cp;
    plane_geometry(d, &Hp, &Wp, &S, &Cp);
    o->P = P;
    if (d->tile_h || d->tile_w) {
        const u32 th = d->tile_h, tw = d->tile_w;
        if (!th || !tw || th > Hp || tw > Wp) fail(HE_EINVAL, "tile must be given in both directions, within the image");
        if ((th % S && th != Hp) || (tw % S && tw != Wp)) fail(HE_EINVAL, "tile sides must be multiples of the stride");
        if ((u64)(th + 2 * P) * (tw + 2 * P) > half)
            fail(HE_EINVAL, "padded tile does not fit a slot row (N/2 positions, N/4 with c_n = 4)");
        o->T_h = th, o->T_w = tw;
    } else {
        choose_tile(half, Hp, Wp, P, S, &o->T_h, &o->T_w);
    }
    o->W_b = o->T_w + 2 * P;
    o->block_slots = (o->T_h + 2 * P) * o->W_b;
    o->blocks_per_row = half / o->block_slots;
    o->n_ty = (Hp + o->T_h - 1) / o->T_h;
    o->n_tx = (Wp + o->T_w - 1) / o->T_w;
    o->units = d->n_images * o->n_ty * o->n_tx;
    u32 per_ct = o->blocks_per_row * (d->c_n == 1 ? 2 : 1);
    o->row_units = (o->units + per_ct - 1) / per_ct;
    o->in_groups = (Cp + d->c_n - 1) / d->c_n;
    o->out_groups = (d->C_out + d->c_n - 1) / d->c_n;
    o->n_ct_in = o->row_units * o->in_groups;
    o->n_ct_out = o->row_units * o->out_groups;
    o->Ho = (Hp - 1) / S + 1;
    o->Wo = (Wp - 1) / S + 1;
    o->scale = d->c_n == 4 ? (4 * p->k4) % p->t : d->c_n == 2 ? (2 * p->k) % p->t : 1;
    std::vector<RotEntry> rl = rotation_list(p, d, *o);
    std::vector<u32> gs;
    for (auto& r : rl)
        if (r.galois != 1) gs.push_back(r.galois);
    std::sort(gs.begin(), gs.end());
    o->n_galois = (u32)(std::unique(gs.begin(), gs.end()) - gs.begin());
}

std::vector<RotEntry> rotation_list(const he_params* p, const he_conv_desc* d, const he_layout& lay) {
    std::vector<RotEntry> out;
    const i64 P = lay.P;
    const u32 ndiag = (d->c_n != 1 && !d->depthwise) ? 2 : 1;
    const u32 swap = 2 * p->N - 1;
    if (d->c_n == 4) {
        // steps 2o for every tap offset o = dy W_b + dx and, unless depthwise (an output class then
        // reads only its own class), the parity-changing steps 2o - 1 and 2o + 1; ascending
        std::vector<i64> steps;
        for (i64 dy = -P; dy <= P; dy++)
            for (i64 dx = -P; dx <= P; dx++) {
                const i64 o = dy * (i64)lay.W_b + dx;
                steps.push_back(2 * o);
                if (!d->depthwise) steps.push_back(2 * o - 1), steps.push_back(2 * o + 1);
            }
        std::sort(steps.begin(), steps.end());
        steps.erase(std::unique(steps.begin(), steps.end()), steps.end());
        for (i64 st : steps) {
            const u32 g = rotation_galois(p, st);
            for (u32 dg = 0; dg < ndiag; dg++)
                out.push_back({~0u, dg, dg ? (u32)((u64)g * swap % (2ULL * p->N)) : g, st});
        }
        return out;
    }
    u32 tap = 0;
    for (i64 dy = -P; dy <= P; dy++)
        for (i64 dx = -P; dx <= P; dx++, tap++) {
            // polyphase planes are read at offsets -1 and 0 only (tap index stays the 3x3 one)
            if (d->polyphase && (dy > 0 || dx > 0)) continue;
            u32 g = rotation_galois(p, dy * (i64)lay.W_b + dx);
            for (u32 dg = 0; dg < ndiag; dg++) {
                u32 gg = dg ? (u32)((u64)g * swap % (2ULL * p->N)) : g;
                out.push_back({tap, dg, gg, dy * (i64)lay.W_b + dx});
            }
        }
    return out;
}
}  // namespace hy

extern "C" int he_layout_for_layer(const he_params* p, const he_conv_desc* d, he_layout* out) {
    return guard([&] {
        if (!p || !d || !out) fail(HE_EINVAL, "null argument");
        compute_layout(p, d, out);
    });
}
extern "C" int he_layer_galois(const he_params* p, const he_conv_desc* d, uint32_t* galois, int cap, int* n) {
    return guard([&] {
        if (!p || !d || !n) fail(HE_EINVAL, "null argument");
        he_layout lay;
        compute_layout(p, d, &lay);
        std::vector<u32> gs;
        for (auto& r : rotation_list(p, d, lay))
            if (r.galois != 1) gs.push_back(r.galois);
        std::sort(gs.begin(), gs.end());
        gs.erase(std::unique(gs.begin(), gs.end()), gs.end());
        *n = (int)gs.size();
        if (galois) {
            if (cap < (int)gs.size()) fail(HE_EINVAL, "galois buffer too small");
            for (size_t i = 0; i < gs.size(); i++) galois[i] = gs[i];
        }
    });
}

// row and position of block-local position (yl, xl) of the u-th tile held by a ciphertext
static void slot_of(const he_conv_desc* d, const he_layout& lay, u32 u, u32 yl, u32 xl, u32* row, u32* pos) {
    u32 B = lay.blocks_per_row, b;
    if (d->c_n == 1) *row = u / B, b = u % B;
    else *row = 0, b = u;
    *pos = b * lay.block_slots + yl * lay.W_b + xl;
}

// flat slot of channel r (0 .. c_n - 1) of a ciphertext at (row, pos): c_n = 1 uses the row,
// c_n = 2 puts channel r in row r, c_n = 4 in row r >> 1 at slot parity r & 1
static u32 flat_slot(const he_conv_desc* d, u32 N, u32 row, u32 pos, u32 r) {
    const u32 half = N / 2;
    if (d->c_n == 1) return row * half + pos;
    if (d->c_n == 2) return r * half + pos;
    return (r >> 1) * half + 2 * pos + (r & 1);
}

extern "C" int he_encrypt_image(const he_params* p, const he_seckey* sk, const he_conv_desc* d, const int64_t* act,
                                uint64_t seed, uint64_t* ct_out) {
    return guard([&] {
        if (!p || !sk || !d || !act || !ct_out) fail(HE_EINVAL, "null argument");
        he_layout lay;
        compute_layout(p, d, &lay);
        const u32 N = p->N, P = lay.P;
        const u32 per_ct = lay.blocks_per_row * (d->c_n == 1 ? 2 : 1);
        u32 Hp, Wp, S, Cplanes;
        plane_geometry(d, &Hp, &Wp, &S, &Cplanes);
        const u32 Cp = Cplanes / (d->polyphase ? 4 : 1);
        // activation of plane channel c at plane position (Y, X): the image itself, or phase
        // (a, b) = (c / Cp) of channel c % Cp at (2Y + a, 2X + b); zero outside the image
        auto A = [&](u32 img, u32 c, i64 Y, i64 X) -> int64_t {
            if (!d->polyphase) return act[(((size_t)img * d->C_in + c) * d->H + Y) * d->W + X];
            const u32 ph = c / Cp, ch = c % Cp;
            const i64 y = 2 * Y + (ph >> 1), x = 2 * X + (ph & 1);
            if (ch >= d->C_in || y >= (i64)d->H || x >= (i64)d->W) return 0;
            return act[(((size_t)img * d->C_in + ch) * d->H + y) * d->W + x];
        };
        std::vector<int64_t> slots((size_t)lay.n_ct_in * N, 0);
        for (u32 unit = 0; unit < lay.units; unit++) {
            u32 ru = unit / per_ct, u = unit % per_ct;
            u32 img = unit / (lay.n_ty * lay.n_tx), rest = unit % (lay.n_ty * lay.n_tx);
            u32 ty = rest / lay.n_tx, tx = rest % lay.n_tx;
            for (u32 yl = 0; yl < lay.T_h + 2 * P; yl++) {
                i64 Y = (i64)ty * lay.T_h + yl - P;
                if (Y < 0 || Y >= (i64)Hp) continue;
                for (u32 xl = 0; xl < lay.W_b; xl++) {
                    i64 X = (i64)tx * lay.T_w + xl - P;
                    if (X < 0 || X >= (i64)Wp) continue;
                    u32 row, pos;
                    slot_of(d, lay, u, yl, xl, &row, &pos);
                    for (u32 j = 0; j < lay.in_groups; j++) {
                        int64_t* sv = slots.data() + (size_t)(ru * lay.in_groups + j) * N;
                        for (u32 r = 0; r < d->c_n; r++) {
                            const u32 c = d->c_n * j + r;
                            if (c < Cplanes) sv[flat_slot(d, N, row, pos, r)] = A(img, c, Y, X);
                        }
                    }
                }
            }
        }
        const size_t ctw = 2ULL * p->L * N;
        parallel_for(lay.n_ct_in, [&](u32 c) {  // ciphertext c draws from its own counter streams
            std::vector<u64> m;
            encode_slots(p, slots.data() + (size_t)c * N, m);
            encrypt_poly(p, sk, m, seed, c, ct_out + c * ctw);
        });
    });
}

extern "C" int he_decrypt_image(const he_params* p, const he_seckey* sk, const he_conv_desc* d, const uint64_t* ct,
                                int unscale, int64_t* out) {
    return guard([&] {
        if (!p || !sk || !d || !ct || !out) fail(HE_EINVAL, "null argument");
        he_layout lay;
        compute_layout(p, d, &lay);
        u32 Hp, Wp, S, Cplanes;
        plane_geometry(d, &Hp, &Wp, &S, &Cplanes);
        const u32 N = p->N, P = lay.P;
        const u32 per_ct = lay.blocks_per_row * (d->c_n == 1 ? 2 : 1);
        const size_t ctw = 2ULL * p->L * N;
        std::vector<int64_t> slots((size_t)lay.n_ct_out * N);
        parallel_for(lay.n_ct_out, [&](u32 c) {
            std::vector<u64> m;
            decrypt_poly(p, sk, ct + c * ctw, m);
            decode_slots(p, m, slots.data() + (size_t)c * N);
        });
        u64 inv = unscale ? p->mod_t.inv(lay.scale % p->t) : 1;
        std::memset(out, 0, sizeof(int64_t) * (size_t)d->n_images * d->C_out * lay.Ho * lay.Wo);
        for (u32 unit = 0; unit < lay.units; unit++) {
            u32 ru = unit / per_ct, u = unit % per_ct;
            u32 img = unit / (lay.n_ty * lay.n_tx), rest = unit % (lay.n_ty * lay.n_tx);
            u32 ty = rest / lay.n_tx, tx = rest % lay.n_tx;
            for (u32 yl = P; yl < P + lay.T_h; yl++) {
                u32 Y = ty * lay.T_h + yl - P;
                if (Y >= Hp || Y % S) continue;
                for (u32 xl = P; xl < P + lay.T_w; xl++) {
                    u32 X = tx * lay.T_w + xl - P;
                    if (X >= Wp || X % S) continue;
                    u32 row, pos;
                    slot_of(d, lay, u, yl, xl, &row, &pos);
                    for (u32 g = 0; g < lay.out_groups; g++) {
                        const int64_t* sv = slots.data() + (size_t)(ru * lay.out_groups + g) * N;
                        auto put = [&](u32 c, int64_t v) {
                            out[(((size_t)img * d->C_out + c) * lay.Ho + Y / S) * lay.Wo + X / S] =
                                (int64_t)p->mod_t.mul((u64)v, inv);
                        };
                        for (u32 r = 0; r < d->c_n; r++)
                            if (d->c_n * g + r < d->C_out) put(d->c_n * g + r, sv[flat_slot(d, N, row, pos, r)]);
                    }
                }
            }
        }
    });
}
