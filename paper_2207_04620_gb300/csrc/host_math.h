// Host-side number theory, randomness and encoding for the hx runtime.
#pragma once
#include <complex>
#include <cstdint>
#include <vector>

namespace hx {

typedef unsigned __int128 u128;

inline uint64_t hmul(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }
uint64_t hpow(uint64_t a, uint64_t e, uint64_t q);
uint64_t hinv(uint64_t a, uint64_t q);  // q prime
bool is_prime_u64(uint64_t n);
// For each size b (in order): largest prime < 2^b, = 1 mod 2N, not yet chosen.
std::vector<uint64_t> choose_primes(int log_n, const std::vector<int> &bits);
// psi = x^((q-1)/2N) for the smallest x >= 2 with psi^N = -1 mod q.
uint64_t find_psi(uint64_t q, int log_n);
uint64_t shoup_companion(uint64_t w, uint64_t q);  // floor(w * 2^64 / q)
uint64_t galois_for_step(int64_t k, int log_n);    // 5^(k mod N/2) mod 2N

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based stream keyed by
// (seed, purpose, a, b): state0 = seed ^ mix64(key + gamma), draw i returns
// mix64(state0 + (i+1)*gamma), key = purpose<<56 | a<<32 | b.
enum Purpose : uint64_t {
    P_SK = 1, P_PK_A = 2, P_PK_E = 3, P_KEY_A = 4, P_KEY_E = 5, P_ENC_V = 6, P_ENC_E0 = 7, P_ENC_E1 = 8, P_SMUDGE = 9,
    P_PCKS_U = 10, P_PCKS_E0 = 11, P_PCKS_E1 = 12,                    // collective key switch
    P_DB_MASK = 13, P_DB_E0 = 14, P_DB_E1 = 15, P_DB_CRP = 16          // collective refresh
};
uint64_t mix64(uint64_t z);
struct Stream {
    uint64_t state;
    Stream(uint64_t seed, uint64_t purpose, uint64_t a, uint64_t b);
    uint64_t next()
    {
        state += 0x9E3779B97F4A7C15ull;
        return mix64(state);
    }
};
// uniform mod q: rejection on bitlen(q) low bits
void sample_uniform(Stream &s, uint64_t q, uint64_t *out, int n);
// {-1,0,1}: draw % 3 with 0->0, 1->1, 2->-1
void sample_ternary(Stream &s, int64_t *out, int n);
// discrete Gaussian by cumulative table on [-B, B], B = floor(6 sigma)
struct GaussianCdt {
    int bound;
    std::vector<uint64_t> th;
    explicit GaussianCdt(double sigma);
    int64_t draw(Stream &s) const;
};

// round half away from zero, evaluated as sign(x) * floor(|x| + 0.5)
double round_half_away(double x);

// Double-double numbers: the unevaluated sum hi + lo of two doubles, about 106 bits
// (Dekker 1971 for the exact product through a fused multiply-add, Knuth's two-sum).
struct DD {
    double hi, lo;
};
DD dd_add(DD a, DD b);
DD dd_mul(DD a, DD b);
DD dd_mul_d(DD a, double b);
// The encoder's rounding rule: hi + lo rounded half away from zero, a value within
// 2^-20 of a half-integer taken as that half-integer.  Throws past 2^62.
int64_t dd_round_coeff(DD x);

// Canonical-embedding encoder/decoder (slot j at zeta^(5^j), zeta = e^(i pi/N)).
// Encoding is exact: coefficient i is scale * (2/N) * sum_j z_j cos(pi (i e_j mod 2N)/N)
// under dd_round_coeff, the sum taken by a double-double FFT of length 2N whose error
// (about 2^-90 relative) lies far inside the rounding rule's band.
struct Encoder {
    int log_n, n;
    std::vector<int64_t> e;  // 5^j mod 2N
    std::vector<DD> roots_re, roots_im;  // e^(-2 pi i k / 2N), k < N, double-double
    std::vector<std::complex<double>> roots;  // the same rounded to double (decoding)
    explicit Encoder(int log_n);
    // m_i = (2/N) sum_j z_j cos(pi (i e_j mod 2N)/N) before the scale, double-double
    void encode_real(const double *slots, size_t count, std::vector<DD> &m) const;
    // coeffs = dd_round_coeff(scale * m)
    void encode(const double *slots, size_t count, double scale, int64_t *coeffs) const;
    // z_j = sum_i c_i zeta^(i e_j) / scale (real part)
    void decode(const int64_t *coeffs, double scale, double *slots, size_t count) const;

  private:
    void fft(std::vector<std::complex<double>> &a, bool inverse) const;
};

} // namespace hx
