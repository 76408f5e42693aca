// Internal declarations shared by the host code (host.cpp) and the device
// code (device.cu) of the library.  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/hyena.h"

namespace hy {

using u64 = uint64_t;
using i64 = int64_t;
using u32 = uint32_t;
using u128 = unsigned __int128;
using i128 = __int128;

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};
[[noreturn]] void fail(int code, const std::string& msg);
void set_last_error(const std::string& msg);

// Runs f, converting exceptions into a status code and the thread-local message.
template <class F>
int guard(F&& f) {
    try {
        f();
        set_last_error("");
        return HE_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return HE_ENOMEM;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return HE_EINVAL;
    }
}

// ------------------------------------------------------------------ modulus
// Barrett constant for x < 2^(s+63), s = bit length of q:
//   mu = floor(2^(s+63) / q),  quotient estimate = mulhi(x >> (s-1), mu),
// which undershoots floor(x/q) by at most 2 (so two conditional subtractions).
struct Modulus {
    u64 q = 0;
    u64 mu = 0;
    u32 sm1 = 0;  // s - 1
    static Modulus make(u64 q);
    u64 reduce(u128 x) const {
        u64 lo = (u64)x, hi = (u64)(x >> 64);
        u64 q1 = (lo >> sm1) | (hi << (64 - sm1));
        u64 q3 = (u64)(((u128)q1 * mu) >> 64);
        u64 r = lo - q3 * q;
        if (r >= q) r -= q;
        if (r >= q) r -= q;
        return r;
    }
    u64 mul(u64 a, u64 b) const { return reduce((u128)a * b); }
    u64 add(u64 a, u64 b) const {
        u64 s = a + b;
        return s >= q ? s - q : s;
    }
    u64 sub(u64 a, u64 b) const { return a >= b ? a - b : a + q - b; }
    u64 pow(u64 a, u64 e) const;
    u64 inv(u64 a) const { return pow(a, q - 2); }
    u64 from_signed(i64 v) const {
        i64 r = v % (i64)q;
        return (u64)(r < 0 ? r + (i64)q : r);
    }
};

inline u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
inline u32 bit_reverse(u32 x, int bits) {
    u32 r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

// Negacyclic NTT on the host with the same ordering as the device kernels:
// Cooley-Tukey, natural input, bit-reversed output; index k holds
// a(psi^(2 rev(k) + 1)).
struct HostNtt {
    int N = 0, logN = 0;
    Modulus m;
    u64 psi = 0;
    std::vector<u64> tw, tw_sh, itw, itw_sh;  // psi^rev(k), psi^-rev(k)
    u64 ninv = 0, ninv_sh = 0;
    void init(int N, u64 q, u64 psi);
    void forward(u64* a) const;
    void inverse(u64* a) const;
};

// Multi-word unsigned integer, little-endian 64-bit words (for CRT lifts).
struct Big {
    std::vector<u64> w;
    static Big from_u64(u64 v) { Big b; b.w = {v}; return b; }
    void trim() { while (w.size() > 1 && w.back() == 0) w.pop_back(); }
    bool is_zero() const { return w.size() == 1 && w[0] == 0; }
};
Big big_mul_u64(const Big& a, u64 b);
Big big_add(const Big& a, const Big& b);
Big big_sub(const Big& a, const Big& b);  // requires a >= b
int big_cmp(const Big& a, const Big& b);
u64 big_mod_u64(const Big& a, u64 m);
double big_log2(const Big& a);
// floor(a / b) for a quotient known to fit in 64 bits
u64 big_div_small_quotient(const Big& a, const Big& b);

// Per-device constant tables of one parameter set.
struct DeviceTables {
    int device = -1;
    u64* tw = nullptr;      // [L][N][2] psi^rev(k) and its Shoup companion
    u64* itw = nullptr;     // [L][N][2] psi^-rev(k) and its Shoup companion
};

}  // namespace hy

struct he_params {
    hy::u32 N = 0, L = 0, logN = 0, w = 0, l = 0;
    hy::u64 t = 0, zeta = 0, h = 0, k = 1;
    hy::i64 kh = 0;
    // c_n = 4: k of the three Walsh-Hadamard patterns and their centred coefficients [3][N]
    // (b = 1, 2, 3: slot parity, row, their product; unscaled +-1 patterns)
    hy::u64 k4 = 1;
    std::vector<hy::i64> pat4;
    std::vector<hy::u64> q, psi;
    std::vector<hy::Modulus> mod;
    std::vector<hy::HostNtt> ntt;  // one per limb
    hy::HostNtt ntt_t;             // mod t with root zeta (slot encoding)
    hy::Modulus mod_t;
    std::vector<hy::u64> delta_mod;  // floor(Q/t) mod q_k
    hy::Big Q, delta;
    std::vector<hy::Big> crt_Qk;     // Q / q_k
    std::vector<hy::u64> crt_inv;    // [(Q/q_k)^-1]_{q_k}
    double log2_delta = 0, est_noise_log2 = 0;
    std::vector<hy::u32> slot_index;  // NTT position of each flat slot
    // device tables, created on first use per device
    mutable std::mutex dev_mu;
    mutable std::vector<hy::DeviceTables*> dev;
    ~he_params();
};

struct he_seckey {
    const he_params* p = nullptr;
    std::vector<hy::i64> s;
    std::vector<hy::u64> s_ntt;  // [L][N]: s in each limb, host NTT form, for the products a*s
};

struct he_galkeys {
    const he_params* p = nullptr;
    std::vector<hy::u32> galois;
    std::vector<std::vector<hy::u64>> keys;  // per element: [L*l][2][L][N] coefficient form
    const std::vector<hy::u64>* find(hy::u32 g) const {
        for (size_t i = 0; i < galois.size(); i++)
            if (galois[i] == g) return &keys[i];
        return nullptr;
    }
};

namespace hy {
// Layout and rotation list of a layer.
struct RotEntry {
    u32 tap, d, galois;
    i64 step;  // left-rotation step before the row swap d (c_n = 4 keys its scalars on it)
};
void compute_layout(const he_params* p, const he_conv_desc* d, he_layout* out);
// plane height, width, stride and channel count the slots of a layer hold (polyphase: the phase planes)
void plane_geometry(const he_conv_desc* d, u32* H, u32* W, u32* S, u32* C_planes);
std::vector<RotEntry> rotation_list(const he_params* p, const he_conv_desc* d, const he_layout& lay);
u32 rotation_galois(const he_params* p, i64 step);
// log2 of the estimated worst output noise (6 sigma + rounding terms).
double estimate_noise_log2(const he_params* p, u32 w, double sum_s0_sq, double sum_s1_sq, double sum_abs_s,
                           bool packed);
// The same for c_n = 4: sum_sq[b] = sum of s_b^2 over a row's terms, out = k4 A0 + sum_b A_b (k4 pattern_b).
double estimate_noise_log2_h4(const he_params* p, u32 w, const double sum_sq[4], double sum_abs_s);
const DeviceTables& device_tables(const he_params* p);
}  // namespace hy
