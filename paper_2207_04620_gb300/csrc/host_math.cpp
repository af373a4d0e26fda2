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

// ---- double-double arithmetic (host code is built with -ffp-contract=off: every operation
// below is rounded once, as written)

static inline DD two_sum(double a, double b)
{
    const double s = a + b, v = s - a;
    return DD{s, (a - (s - v)) + (b - v)};
}

static inline DD fast_two_sum(double a, double b)  // |a| >= |b|
{
    const double s = a + b;
    return DD{s, b - (s - a)};
}

static inline DD two_prod(double a, double b)
{
    const double p = a * b;
    return DD{p, std::fma(a, b, -p)};  // the exact error of the product
}

DD dd_add(DD a, DD b)
{
    DD s = two_sum(a.hi, b.hi);
    const DD t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(s.hi, s.lo + t.lo);
}

DD dd_mul(DD a, DD b)
{
    const DD p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, p.lo + (a.hi * b.lo + a.lo * b.hi));
}

DD dd_mul_d(DD a, double b)
{
    const DD p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, p.lo + a.lo * b);
}

static DD dd_div_d(DD a, double b)
{
    const double q1 = a.hi / b;
    const DD p = two_prod(q1, b);
    const double r = ((a.hi - p.hi) - p.lo) + a.lo;
    return fast_two_sum(q1, r / b);
}

int64_t dd_round_coeff(DD x)
{
    if (!(std::fabs(x.hi) < 4611686018427387904.0)) throw std::runtime_error("encoded coefficient exceeds 2^62");
    // integer parts of both words (each exact), and what is left of each
    const double i1 = std::nearbyint(x.hi), i2 = std::nearbyint(x.lo);
    const double f = (x.hi - i1) + (x.lo - i2);  // |f| <= 1
    const int64_t base = (int64_t)i1 + (int64_t)i2;
    const double band = 0x1p-20;
    int64_t c = base;
    if (std::fabs(std::fabs(f) - 0.5) <= band) {
        // the half-integer base +- 1/2, rounded away from zero
        const bool positive = f > 0 ? base >= 0 : base > 0;
        c = f > 0 ? (positive ? base + 1 : base) : (positive ? base : base - 1);
    } else if (f > 0.5) {
        c = base + 1;
    } else if (f < -0.5) {
        c = base - 1;
    }
    if (c >= ((int64_t)1 << 62) || c <= -((int64_t)1 << 62)) throw std::runtime_error("encoded coefficient exceeds 2^62");
    return c;
}

// cos and sin of pi * a / b, 0 <= a/b <= 1/4, in double-double: Taylor series of the angle
// pi*a/b (pi as the double-double 0x1.921fb54442d18p+1 + 0x1.1a62633145c07p-53)
static void dd_cos_sin_pi(int64_t a, int64_t b, DD &c, DD &s)
{
    const DD pi{0x1.921fb54442d18p+1, 0x1.1a62633145c07p-53};
    const DD phi = dd_div_d(dd_mul_d(pi, (double)a), (double)b);
    const DD phi2 = dd_mul(phi, phi);
    DD tc{1.0, 0.0}, ts = phi;
    c = tc;
    s = ts;
    for (int k = 0; k < 40; k++) {
        tc = dd_div_d(dd_mul(tc, phi2), -(double)((2 * k + 1) * (2 * k + 2)));
        ts = dd_div_d(dd_mul(ts, phi2), -(double)((2 * k + 2) * (2 * k + 3)));
        c = dd_add(c, tc);
        s = dd_add(s, ts);
        if (std::fabs(tc.hi) < 0x1p-112 && std::fabs(ts.hi) < 0x1p-112) break;
    }
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
    // e^(-2 pi i k / 2N) = cos(pi k/N) - i sin(pi k/N) for k < N, from the angles in [0, pi/4]
    // (k = N/4 is pi/4) by the symmetries of cos and sin
    const int m8 = n / 4;
    std::vector<DD> tc(m8 + 1), ts(m8 + 1);
    for (int j = 0; j <= m8; j++) dd_cos_sin_pi(j, n, tc[j], ts[j]);
    auto neg = [](DD x) { return DD{-x.hi, -x.lo}; };
    roots_re.resize(n);
    roots_im.resize(n);
    roots.resize(n);
    for (int k = 0; k < n; k++) {
        DD c, si;
        if (k <= m8) {
            c = tc[k];
            si = ts[k];
        } else if (k <= 2 * m8) {  // pi/2 - angle
            c = ts[2 * m8 - k];
            si = tc[2 * m8 - k];
        } else if (k <= 3 * m8) {  // pi/2 + angle
            c = neg(ts[k - 2 * m8]);
            si = tc[k - 2 * m8];
        } else {  // pi - angle
            c = neg(tc[4 * m8 - k]);
            si = ts[4 * m8 - k];
        }
        roots_re[k] = c;
        roots_im[k] = neg(si);
        roots[k] = std::complex<double>(c.hi, -si.hi);
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

void Encoder::encode_real(const double *slots, size_t count, std::vector<DD> &m) const
{
    // radix-2 decimation in time over the slots scattered to exponents e_j and 2N - e_j (the
    // conjugate of a real slot), in bit-reversed order; complex values as double-double pairs.
    // Every exponent that holds a slot is odd, and bit reversal sends the even ones (zeros) to the
    // first half, which stays zero until the last stage; that stage gives A_i = w_i B_i (i < N)
    // from the second half B.  So only the second half is transformed, and the last stage is
    // folded into the read-out (adding a zero returns the other operand exactly: the values are
    // the full transform's).
    const int len = 2 * n, bits = log_n + 1;
    std::vector<DD> re(n, DD{0.0, 0.0}), im(n, DD{0.0, 0.0});  // positions n .. 2n - 1
    auto brv = [&](int x) {
        int r = 0;
        for (int b = 0; b < bits; b++) r |= ((x >> b) & 1) << (bits - 1 - b);
        return r;
    };
    for (size_t j = 0; j < (size_t)(n / 2); j++) {
        const double z = j < count ? slots[j] : 0.0;
        re[brv((int)e[j]) - n] = DD{z, 0.0};
        re[brv((int)((len - e[j]) % len)) - n] = DD{z, 0.0};
    }
    for (int half = 1; half < n; half <<= 1) {
        const int step = n / half;  // root index stride: e^(-2 pi i k / (2 half)) = roots[k * step]
        for (int i = 0; i < n; i += 2 * half)
            for (int k = 0; k < half; k++) {
                const DD wr = roots_re[(size_t)k * step], wi = roots_im[(size_t)k * step];
                const DD vr = re[i + k + half], vi = im[i + k + half];
                const DD vw = dd_mul(vi, wi);
                const DD tr = dd_add(dd_mul(vr, wr), DD{-vw.hi, -vw.lo});
                const DD ti = dd_add(dd_mul(vr, wi), dd_mul(vi, wr));
                const DD ur = re[i + k], ui = im[i + k];
                re[i + k] = dd_add(ur, tr);
                im[i + k] = dd_add(ui, ti);
                re[i + k + half] = dd_add(ur, DD{-tr.hi, -tr.lo});
                im[i + k + half] = dd_add(ui, DD{-ti.hi, -ti.lo});
            }
    }
    m.resize(n);
    const double inv_n = 1.0 / n;  // a power of two: exact
    for (int i = 0; i < n; i++) {
        const DD vw = dd_mul(im[i], roots_im[i]);
        const DD r = dd_add(dd_mul(re[i], roots_re[i]), DD{-vw.hi, -vw.lo});  // Re(w_i B_i)
        m[i] = DD{r.hi * inv_n, r.lo * inv_n};
    }
}

void Encoder::encode(const double *slots, size_t count, double scale, int64_t *coeffs) const
{
    std::vector<DD> m;
    encode_real(slots, count, m);
    for (int i = 0; i < n; i++) coeffs[i] = dd_round_coeff(dd_mul_d(m[i], scale));
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
