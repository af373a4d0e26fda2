#include "host_math.h"

#include <cmath>
#include <stdexcept>

namespace hx {

uint64_t hpow(uint64_t a, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = hmul(r, a, q);
        a = hmul(a, a, q);
        e >>= 1;
    }
    return r;
}

uint64_t hinv(uint64_t a, uint64_t q) { return hpow(a % q, q - 2, q); }

bool is_prime_u64(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t p : bases)
        if (n % p == 0) return n == p;
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        s++;
    }
    for (uint64_t a : bases) {
        uint64_t x = hpow(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; r++) {
            x = hmul(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

std::vector<uint64_t> choose_primes(int log_n, const std::vector<int> &bits)
{
    const uint64_t two_n = 2ull << log_n;
    std::vector<uint64_t> out;
    for (int b : bits) {
        uint64_t c = (1ull << b) - two_n + 1;
        for (;;) {
            bool used = false;
            for (uint64_t x : out) used |= (x == c);
            if (!used && is_prime_u64(c)) break;
            if (c <= two_n + two_n) throw std::runtime_error("no suitable prime");
            c -= two_n;
        }
        out.push_back(c);
    }
    return out;
}

uint64_t find_psi(uint64_t q, int log_n)
{
    const uint64_t n = 1ull << log_n;
    const uint64_t e = (q - 1) / (2 * n);
    for (uint64_t x = 2;; x++) {
        uint64_t psi = hpow(x, e, q);
        if (hpow(psi, n, q) == q - 1) return psi;
    }
}

uint64_t shoup_companion(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

uint64_t galois_for_step(int64_t k, int log_n)
{
    const int64_t s = 1ll << (log_n - 1);
    int64_t r = ((k % s) + s) % s;
    return hpow(5, (uint64_t)r, 2ull << log_n);
}

uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

Stream::Stream(uint64_t seed, uint64_t purpose, uint64_t a, uint64_t b)
{
    const uint64_t key = ((purpose & 0xFF) << 56) | ((a & 0xFFFFFF) << 32) | (b & 0xFFFFFFFFull);
    state = seed ^ mix64(key + 0x9E3779B97F4A7C15ull);
}

void sample_uniform(Stream &s, uint64_t q, uint64_t *out, int n)
{
    int bl = 64 - __builtin_clzll(q);
    const uint64_t mask = bl >= 64 ? ~0ull : ((1ull << bl) - 1);
    for (int i = 0; i < n;) {
        uint64_t r = s.next() & mask;
        if (r < q) out[i++] = r;
    }
}

void sample_ternary(Stream &s, int64_t *out, int n)
{
    for (int i = 0; i < n; i++) {
        uint64_t r = s.next() % 3;
        out[i] = r == 2 ? -1 : (int64_t)r;
    }
}

GaussianCdt::GaussianCdt(double sigma)
{
    bound = (int)std::floor(6.0 * sigma);
    const double two_s2 = 2.0 * sigma * sigma;
    std::vector<double> w;
    for (int k = -bound; k <= bound; k++) w.push_back(std::exp(-(double)(k * k) / two_s2));
    double total = 0.0;
    for (double x : w) total += x;
    double cum = 0.0;
    for (double x : w) {
        cum += x;
        th.push_back((uint64_t)std::floor((cum / total) * 9223372036854775808.0));
    }
}

int64_t GaussianCdt::draw(Stream &s) const
{
    const uint64_t r = s.next() >> 1;
    int idx = 0;
    const int last = 2 * bound;
    while (idx < last && r >= th[idx]) idx++;
    return (int64_t)idx - bound;
}

double round_half_away(double x)
{
    double a = std::floor(std::fabs(x) + 0.5);
    return x < 0 ? -a : a;
}

Encoder::Encoder(int ln) : log_n(ln), n(1 << ln)
{
    const int s = n / 2;
    e.resize(s);
    int64_t v = 1;
    for (int j = 0; j < s; j++) {
        e[j] = v;
        v = v * 5 % (2 * n);
    }
    roots.resize(n);  // half of the 2N-th roots suffice for a 2N-point FFT
    for (int k = 0; k < n; k++) {
        const double ang = -2.0 * M_PI * (double)k / (double)(2 * n);
        roots[k] = std::complex<double>(std::cos(ang), std::sin(ang));
    }
}

// iterative radix-2 FFT of length 2N: A_k = sum_i a_i w^(ik), w = e^(-+2 pi i / 2N)
void Encoder::fft(std::vector<std::complex<double>> &a, bool inverse) const
{
    const int m = 2 * n;
    for (int i = 1, j = 0; i < m; i++) {
        int bit = m >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (int len = 2; len <= m; len <<= 1) {
        const int step = m / len;
        for (int i = 0; i < m; i += len)
            for (int k = 0; k < len / 2; k++) {
                std::complex<double> w = roots[k * step];
                if (inverse) w = std::conj(w);
                std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

void Encoder::encode(const double *slots, size_t count, double scale, int64_t *coeffs) const
{
    const int m = 2 * n;
    std::vector<std::complex<double>> big(m);
    for (size_t j = 0; j < (size_t)(n / 2); j++) {
        const double z = j < count ? slots[j] : 0.0;
        big[e[j]] = z;
        big[(m - e[j]) % m] = z;  // conjugate of a real slot
    }
    fft(big, false);
    for (int i = 0; i < n; i++) {
        const double v = round_half_away(big[i].real() / n * scale);
        if (!(std::fabs(v) < 4611686018427387904.0)) throw std::runtime_error("encoded coefficient exceeds 2^62");
        coeffs[i] = (int64_t)v;
    }
}

void Encoder::decode(const int64_t *coeffs, double scale, double *slots, size_t count) const
{
    const int m = 2 * n;
    std::vector<std::complex<double>> big(m);
    for (int i = 0; i < n; i++) big[i] = (double)coeffs[i];
    fft(big, true);  // sum_i c_i e^(+2 pi i ik / 2N) = sum_i c_i zeta^(ik)
    for (size_t j = 0; j < count && j < (size_t)(n / 2); j++) slots[j] = big[e[j]].real() / scale;
}

} // namespace hx
