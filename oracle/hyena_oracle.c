/*
 * Plain, slow CPU oracle for BFV homomorphic convolution with Walsh-Hadamard
 * output-channel packing ("Hyena", arXiv 2311.12519).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no source, header, table or helper with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Style: every modular product is a full 128-bit product followed by `%`;
 * every sum is reduced immediately (eager reduction).  No Montgomery, Barrett,
 * Shoup, lazy accumulation, blocking or reordering: the point is that each
 * function can be checked against its definition by eye.
 *
 * Polynomials live in R_q = Z_q[X]/(X^N + 1) (Sec. 2.3); a ciphertext is the
 * pair (c0, c1) stored as u64[2][L][N]: polynomial, RNS limb q_k, coefficient.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* modular helpers (q < 2^62)                                          */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + q - (b % q)) % q); }
static u64 powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}
/* inverse by Fermat (q prime) */
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }
/* signed integer -> residue in [0, q) */
static u64 lift(i64 v, u64 q) {
    i64 r = v % (i64)q;
    if (r < 0) r += (i64)q;
    return (u64)r;
}

/* ------------------------------------------------------------------ */
/* Counter-based random numbers: SplitMix64 (Steele, Lea and Flood,    */
/* OOPSLA 2014).  The state advances by the golden gamma; the output   */
/* is the state passed through the published 64-bit finaliser.         */
/* ------------------------------------------------------------------ */
#define SM_GAMMA 0x9E3779B97F4A7C15ULL

static u64 sm_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* The n-th output (n = 0, 1, ...) of SplitMix64 whose state starts at `key`. */
u64 orc_splitmix_at(u64 key, u64 n) { return sm_mix(key + SM_GAMMA * (n + 1)); }

/* Stream key for (seed, tag, a, b): three chained SplitMix64 look-ups. */
u64 orc_stream_key(u64 seed, u64 tag, u64 a, u64 b) {
    u64 k = orc_splitmix_at(seed, tag);
    k = orc_splitmix_at(k, a);
    return orc_splitmix_at(k, b);
}

typedef struct { u64 key; u64 ctr; } rng_t;
static u64 rng_next(rng_t* r) { return orc_splitmix_at(r->key, r->ctr++); }

/* Uniform integer in [0, m): draw x, reject while x < (2^64 mod m), return x mod m. */
static u64 rng_below(rng_t* r, u64 m) {
    u64 lim = (0 - m) % m; /* = 2^64 mod m */
    for (;;) {
        u64 x = rng_next(r);
        if (x >= lim) return x % m;
    }
}
/* Bernoulli(n/d), 0 <= n <= d. */
static int bern(rng_t* r, u64 n, u64 d) { return rng_below(r, d) < n; }

/*
 * Exact Bernoulli(exp(-n/d)) from Canonne, Kamath and Steinke, "The Discrete
 * Gaussian for Differential Privacy" (2020), Algorithm 1: for gamma <= 1 run
 * the alternating-series loop; for gamma > 1 take floor(gamma) draws of
 * Bernoulli(exp(-1)) and one of Bernoulli(exp(-frac(gamma))).
 */
static int bern_exp_small(rng_t* r, u64 n, u64 d) { /* n <= d */
    u64 K = 1;
    while (bern(r, n, d * K)) K++;
    return (int)(K & 1);
}
static int bern_exp(rng_t* r, u64 n, u64 d) {
    if (n <= d) return bern_exp_small(r, n, d); /* gamma in [0, 1] */
    u64 whole = n / d;
    for (u64 i = 0; i < whole; i++)
        if (!bern_exp_small(r, 1, 1)) return 0;
    return bern_exp_small(r, n % d, d);
}
/* Discrete Laplace with integer scale s (same paper, Algorithm 2). */
static i64 dlaplace(rng_t* r, u64 s) {
    for (;;) {
        u64 U = rng_below(r, s);
        if (!bern_exp(r, U, s)) continue;
        u64 V = 0;
        while (bern_exp(r, 1, 1)) V++;
        u64 X = U + s * V;
        int B = bern(r, 1, 2);
        if (B && X == 0) continue;
        return B ? -(i64)X : (i64)X;
    }
}
/*
 * Discrete Gaussian with variance sig2 = sn/sd (same paper, Algorithm 3),
 * truncated to |e| <= bound by resampling (B-bounded, B = 10 sigma, Sec. 2.3).
 */
static i64 dgauss(rng_t* r, u64 sn, u64 sd, i64 bound) {
    /* s = floor(sigma) + 1 */
    u64 s = 1;
    while ((s * s) * sd <= sn) s++;
    for (;;) {
        i64 Y = dlaplace(r, s);
        u64 aY = (u64)(Y < 0 ? -Y : Y);
        /* gamma = (|Y| - sigma^2/s)^2 / (2 sigma^2) = (|Y| s sd - sn)^2 / (2 s^2 sd sn) */
        i64 diff = (i64)(aY * s * sd) - (i64)sn;
        u64 num = (u64)(diff < 0 ? -diff : diff);
        num = num * num;
        u64 den = 2 * s * s * sd * sn;
        if (!bern_exp(r, num, den)) continue;
        if (Y > bound || Y < -bound) continue;
        return Y;
    }
}

/* ternary coefficient n of the stream: (x mod 3) - 1 */
void orc_sample_ternary(u64 key, int N, i64* out) {
    for (int n = 0; n < N; n++) out[n] = (i64)(orc_splitmix_at(key, (u64)n) % 3) - 1;
}
/* uniform residues mod q[k] for L limbs: coefficient (k, n) from draws 2(kN+n), 2(kN+n)+1 */
void orc_sample_uniform(u64 key, int L, int N, const u64* q, u64* out) {
    for (int k = 0; k < L; k++)
        for (int n = 0; n < N; n++) {
            u64 idx = 2 * ((u64)k * (u64)N + (u64)n);
            u128 x = ((u128)orc_splitmix_at(key, idx) << 64) | orc_splitmix_at(key, idx + 1);
            out[(size_t)k * N + n] = (u64)(x % q[k]);
        }
}
/* discrete Gaussian coefficient n: its own stream keyed by draw n of `key` */
void orc_sample_gauss(u64 key, int N, u64 sn, u64 sd, i64 bound, i64* out) {
    for (int n = 0; n < N; n++) {
        rng_t r = {orc_splitmix_at(key, (u64)n), 0};
        out[n] = dgauss(&r, sn, sd, bound);
    }
}

/* ------------------------------------------------------------------ */
/* Negacyclic NTT, natural order: A[k] = a(psi^(2k+1)), k = 0..N-1,    */
/* psi a primitive 2N-th root of unity mod q (needs q = 1 mod 2N).     */
/* Computed as a cyclic DFT with omega = psi^2 of (a_i psi^i), by the  */
/* iterative radix-2 Cooley-Tukey FFT with an input bit reversal.      */
/* ------------------------------------------------------------------ */
static void bitrev_permute(u64* a, int N) {
    for (int i = 1, j = 0; i < N; i++) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}
static void cyclic_dft(u64* a, int N, u64 q, u64 omega) {
    bitrev_permute(a, N);
    for (int len = 2; len <= N; len <<= 1) {
        u64 wl = powmod(omega, (u64)(N / len), q);
        for (int i = 0; i < N; i += len) {
            u64 w = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j];
                u64 v = mulmod(a[i + j + len / 2], w, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                w = mulmod(w, wl, q);
            }
        }
    }
}
void orc_ntt_fwd(u64* a, int N, u64 q, u64 psi) {
    u64 p = 1;
    for (int i = 0; i < N; i++) { a[i] = mulmod(a[i], p, q); p = mulmod(p, psi, q); }
    cyclic_dft(a, N, q, mulmod(psi, psi, q));
}
void orc_ntt_inv(u64* a, int N, u64 q, u64 psi) {
    u64 psi_inv = invmod(psi, q);
    cyclic_dft(a, N, q, mulmod(psi_inv, psi_inv, q));
    u64 ninv = invmod((u64)N, q);
    u64 p = ninv;
    for (int i = 0; i < N; i++) { a[i] = mulmod(a[i], p, q); p = mulmod(p, psi_inv, q); }
}

/* c = a * b in Z_q[X]/(X^N+1), by NTT, pointwise product, inverse NTT */
void orc_negacyclic_mul(const u64* a, const u64* b, u64* c, int N, u64 q, u64 psi) {
    u64* ta = (u64*)malloc(sizeof(u64) * (size_t)N);
    u64* tb = (u64*)malloc(sizeof(u64) * (size_t)N);
    for (int i = 0; i < N; i++) { ta[i] = a[i] % q; tb[i] = b[i] % q; }
    orc_ntt_fwd(ta, N, q, psi);
    orc_ntt_fwd(tb, N, q, psi);
    for (int i = 0; i < N; i++) c[i] = mulmod(ta[i], tb[i], q);
    orc_ntt_inv(c, N, q, psi);
    free(ta);
    free(tb);
}

/* sigma_g(a)(X) = a(X^g) for odd g: coefficient i moves to i*g mod 2N, negated past N. */
void orc_automorphism(const u64* a, u64* out, int N, u64 q, u64 g) {
    u64 M = 2 * (u64)N;
    for (int i = 0; i < N; i++) {
        u64 j = ((u64)i * g) % M;
        if (j < (u64)N) out[j] = a[i] % q;
        else out[j - N] = submod(0, a[i], q);
    }
}

/* ------------------------------------------------------------------ */
/* BFV symmetric encryption in RNS form (Sec. 2.3):                   */
/*   c0 = [Delta m + a s + e]_q,  c1 = [-a]_q,  Delta = floor(q/t).   */
/* delta_mod[k] = Delta mod q_k; m has entries in [0, t).             */
/* ------------------------------------------------------------------ */
void orc_encrypt(const u64* m, const i64* s, const u64* a, const i64* e, const u64* delta_mod,
                 const u64* q, const u64* psi, int L, int N, u64* ct) {
    u64* sk = (u64*)malloc(sizeof(u64) * (size_t)N);
    u64* as = (u64*)malloc(sizeof(u64) * (size_t)N);
    for (int k = 0; k < L; k++) {
        for (int n = 0; n < N; n++) sk[n] = lift(s[n], q[k]);
        orc_negacyclic_mul(a + (size_t)k * N, sk, as, N, q[k], psi[k]);
        u64* c0 = ct + (size_t)k * N;
        u64* c1 = ct + (size_t)(L + k) * N;
        for (int n = 0; n < N; n++) {
            u64 v = mulmod(delta_mod[k], m[n], q[k]);
            v = addmod(v, as[n], q[k]);
            v = addmod(v, lift(e[n], q[k]), q[k]);
            c0[n] = v;
            c1[n] = submod(0, a[(size_t)k * N + n], q[k]);
        }
    }
    free(sk);
    free(as);
}

/* [c0 + c1 s]_{q_k} for each limb (decryption before the CRT and the rounding) */
void orc_dot_secret(const u64* ct, const i64* s, const u64* q, const u64* psi, int L, int N, u64* out) {
    u64* sk = (u64*)malloc(sizeof(u64) * (size_t)N);
    u64* cs = (u64*)malloc(sizeof(u64) * (size_t)N);
    for (int k = 0; k < L; k++) {
        for (int n = 0; n < N; n++) sk[n] = lift(s[n], q[k]);
        orc_negacyclic_mul(ct + (size_t)(L + k) * N, sk, cs, N, q[k], psi[k]);
        for (int n = 0; n < N; n++) out[(size_t)k * N + n] = addmod(ct[(size_t)k * N + n], cs[n], q[k]);
    }
    free(sk);
    free(cs);
}

/* ------------------------------------------------------------------ */
/* Key switching with a decomposition base 2^w (Sec. 2.3, Rotation).   */
/* Gadget: limb i, digit j has g_ij = 2^(w j) (q/q_i)[(q/q_i)^-1]_{q_i},*/
/* so g_ij = 2^(w j) mod q_i and 0 mod q_k for k != i.                 */
/* ------------------------------------------------------------------ */

/*
 * Galois key for element g (switches sigma_g(s) back to s).  For each digit
 * (i, j), index dd = i*l + j:  b = -a s + e + g_ij sigma_g(s),  key = (b, a).
 * a_all: uniform residues [L*l][L][N]; e_all: errors [L*l][N].
 * Output ksk: [L*l][2][L][N], coefficient form.
 */
void orc_galois_key(const i64* s, u64 g, const u64* a_all, const i64* e_all, const u64* q, const u64* psi,
                    int L, int N, int w, int l, u64* ksk) {
    u64* sk = (u64*)malloc(sizeof(u64) * (size_t)N);
    u64* sg = (u64*)malloc(sizeof(u64) * (size_t)N);
    u64* as = (u64*)malloc(sizeof(u64) * (size_t)N);
    for (int i = 0; i < L; i++)
        for (int j = 0; j < l; j++) {
            int dd = i * l + j;
            const u64* a = a_all + (size_t)dd * L * N;
            const i64* e = e_all + (size_t)dd * N;
            u64* b_out = ksk + ((size_t)dd * 2 + 0) * L * N;
            u64* a_out = ksk + ((size_t)dd * 2 + 1) * L * N;
            for (int k = 0; k < L; k++) {
                for (int n = 0; n < N; n++) sk[n] = lift(s[n], q[k]);
                orc_negacyclic_mul(a + (size_t)k * N, sk, as, N, q[k], psi[k]);
                orc_automorphism(sk, sg, N, q[k], g);
                u64 gij = (k == i) ? powmod(2, (u64)w * (u64)j, q[k]) : 0;
                for (int n = 0; n < N; n++) {
                    u64 v = submod(0, as[n], q[k]);
                    v = addmod(v, lift(e[n], q[k]), q[k]);
                    v = addmod(v, mulmod(gij, sg[n], q[k]), q[k]);
                    b_out[(size_t)k * N + n] = v;
                    a_out[(size_t)k * N + n] = a[(size_t)k * N + n] % q[k];
                }
            }
        }
    free(sk); free(sg); free(as);
}

/*
 * Hoisting, step 1 (done once per ciphertext): split [c1]_{q_i} into l digits
 * base 2^w.  digits: [L*l][N], digit dd = i*l + j = ((c1_i >> w j) & (2^w - 1)).
 */
void orc_decompose(const u64* c1, int L, int N, int w, int l, u64* digits) {
    u64 mask = (w >= 64) ? ~0ULL : ((1ULL << w) - 1);
    for (int i = 0; i < L; i++)
        for (int j = 0; j < l; j++)
            for (int n = 0; n < N; n++) {
                u64 x = c1[(size_t)i * N + n];
                u64 sh = (u64)w * (u64)j;
                digits[((size_t)i * l + j) * N + n] = (sh >= 64) ? 0 : ((x >> sh) & mask);
            }
}

/*
 * Hoisting, step 2 (once per rotation): apply sigma_g to c0 and to every
 * digit polynomial, then multiply the rotated digits by the Galois key and sum:
 *   c0' = sigma(c0) + sum_dd sigma(d_dd) * b_dd,   c1' = sum_dd sigma(d_dd) * a_dd.
 * ct: [2][L][N]; digits from orc_decompose; ksk from orc_galois_key; out: [2][L][N].
 */
void orc_rotate_hoisted(const u64* ct, const u64* digits, const u64* ksk, u64 g, const u64* q, const u64* psi,
                        int L, int N, int l, u64* out) {
    u64* dk = (u64*)malloc(sizeof(u64) * (size_t)N);
    u64* sd = (u64*)malloc(sizeof(u64) * (size_t)N);
    u64* pr = (u64*)malloc(sizeof(u64) * (size_t)N);
    for (int k = 0; k < L; k++) {
        orc_automorphism(ct + (size_t)k * N, out + (size_t)k * N, N, q[k], g);
        memset(out + (size_t)(L + k) * N, 0, sizeof(u64) * (size_t)N);
    }
    for (int dd = 0; dd < L * l; dd++) {
        for (int k = 0; k < L; k++) {
            for (int n = 0; n < N; n++) dk[n] = digits[(size_t)dd * N + n] % q[k];
            orc_automorphism(dk, sd, N, q[k], g);
            for (int p = 0; p < 2; p++) {
                const u64* key = ksk + ((size_t)dd * 2 + p) * L * N + (size_t)k * N;
                orc_negacyclic_mul(sd, key, pr, N, q[k], psi[k]);
                u64* o = out + ((size_t)p * L + k) * N;
                for (int n = 0; n < N; n++) o[n] = addmod(o[n], pr[n], q[k]);
            }
        }
    }
    free(dk); free(sd); free(pr);
}

/*
 * acc += s * x (mod q_k) for a [2][L][N] ciphertext x and a signed integer s
 * (CMult followed by HAdd, both reduced at once: the eager form of Sec. 3.2.2).
 */
void orc_cmult_add(u64* acc, const u64* x, i64 s, const u64* q, int L, int N) {
    for (int p = 0; p < 2; p++)
        for (int k = 0; k < L; k++) {
            u64 sk = lift(s, q[k]);
            u64* a = acc + ((size_t)p * L + k) * N;
            const u64* b = x + ((size_t)p * L + k) * N;
            for (int n = 0; n < N; n++) a[n] = addmod(a[n], mulmod(sk, b[n], q[k]), q[k]);
        }
}

/* out = ct * pt per limb (PMult, Sec. 2.3); pt given as centred integers. */
void orc_pmult(const u64* ct, const i64* pt, const u64* q, const u64* psi, int L, int N, u64* out) {
    u64* pk = (u64*)malloc(sizeof(u64) * (size_t)N);
    for (int k = 0; k < L; k++) {
        for (int n = 0; n < N; n++) pk[n] = lift(pt[n], q[k]);
        for (int p = 0; p < 2; p++)
            orc_negacyclic_mul(ct + ((size_t)p * L + k) * N, pk, out + ((size_t)p * L + k) * N, N, q[k], psi[k]);
    }
    free(pk);
}
