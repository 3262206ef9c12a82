// Floating-point operation count of the oracle's time step: the oracle's own C
// source (evlbm_oracle.c), compiled unchanged as C++ with every `double` replaced
// by a type that counts each +, -, *, / (compound assignments included; negation,
// comparisons and copies are not operations).  TEST INFRASTRUCTURE ONLY, like the
// rest of this directory.
//
// Usage: flopcount Q thermal eos force_form nx ny nz   (or: flopcount selftest)
// Prints "<flops of 1 step> <flops of 2 steps> <nodes>"; the difference is the cost
// of one step (setup work inside orc_step, such as the frozen temperature copy of an
// isothermal run, cancels), and dividing it by the node count gives the operations
// per lattice update of Eq. (pre_LBM) with every stage of the oracle.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <math.h>       // the oracle's own headers, included before `double` is redefined
#include <stdlib.h>
#include <string.h>

static unsigned long long g_ops = 0;

struct CountedDouble {
    double v;
    CountedDouble() = default;
    CountedDouble(double x) : v(x) {}
    CountedDouble(int x) : v(x) {}
    CountedDouble(long x) : v((double)x) {}
    CountedDouble &operator+=(CountedDouble o) { ++g_ops; v += o.v; return *this; }
    CountedDouble &operator-=(CountedDouble o) { ++g_ops; v -= o.v; return *this; }
    CountedDouble &operator*=(CountedDouble o) { ++g_ops; v *= o.v; return *this; }
    CountedDouble &operator/=(CountedDouble o) { ++g_ops; v /= o.v; return *this; }
};
using CD = CountedDouble;
inline CD operator+(CD a, CD b) { ++g_ops; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { ++g_ops; return CD(a.v - b.v); }
inline CD operator*(CD a, CD b) { ++g_ops; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { ++g_ops; return CD(a.v / b.v); }
inline CD operator-(CD a) { return CD(-a.v); }
inline CD operator+(CD a) { return a; }
inline bool operator<(CD a, CD b) { return a.v < b.v; }
inline bool operator>(CD a, CD b) { return a.v > b.v; }
inline bool operator<=(CD a, CD b) { return a.v <= b.v; }
inline bool operator>=(CD a, CD b) { return a.v >= b.v; }
inline bool operator==(CD a, CD b) { return a.v == b.v; }
inline bool operator!=(CD a, CD b) { return a.v != b.v; }

// C's implicit conversion of malloc's void * (and of NULL) to any object pointer.
struct AnyPtr {
    void *p;
    template <class T> operator T *() const { return static_cast<T *>(p); }
};
static AnyPtr any_malloc(size_t n) { return AnyPtr{std::malloc(n)}; }

#define malloc(n) any_malloc(n)
#undef NULL
#define NULL (AnyPtr{nullptr})
#define double CountedDouble
#include "evlbm_oracle.c"
#undef double
#undef malloc

int main(int argc, char **argv)
{
    if (argc == 2 && std::strcmp(argv[1], "selftest") == 0) {   // 4 + 2 operations
        CD a(1.5), b(2.0), c(0.25), d(4.0), e(1.0), x(3.0);
        CD y = (a * b + c) / d - e;
        x += y;
        x *= CD(2.0);
        x = -x;
        std::printf("%llu %.17g\n", g_ops, x.v);
        return 0;
    }
    if (argc != 8) {
        std::fprintf(stderr, "usage: flopcount Q thermal eos force_form nx ny nz\n");
        return 2;
    }
    orc_params p;
    std::memset(&p, 0, sizeof p);
    p.Q = std::atoi(argv[1]);
    p.thermal = std::atoi(argv[2]);
    p.eos = std::atoi(argv[3]);
    p.force_form = std::atoi(argv[4]);
    p.nx = std::atoi(argv[5]);
    p.ny = std::atoi(argv[6]);
    p.nz = std::atoi(argv[7]);
    p.a = 0.1;
    p.b = 4.0;
    p.R = 1.0;
    p.kappa = 0.1;
    p.tau = 0.3;
    p.lambda = 1.0;
    const long N = (long)p.nx * p.ny * p.nz;
    const int D = p.Q == 9 ? 2 : 3;
    CD *rho = new CD[N], *u = new CD[3 * N], *T = new CD[N];
    CD *f = new CD[(size_t)p.Q * N], *g = new CD[(size_t)p.Q * N];
    for (long n = 0; n < N; ++n) {           // a smooth, physical state (liquid-like density)
        rho[n] = CD(0.2 + 0.01 * (double)(n % 7) / 7.0);
        T[n] = CD(0.008);
        for (int a = 0; a < D; ++a) u[a * N + n] = CD(0.01 * (double)((n + a) % 5) / 5.0);
    }
    unsigned long long ops[2];
    for (int k = 0; k < 2; ++k) {
        if (orc_init(&p, rho, u, T, f, g)) return 1;
        g_ops = 0;
        if (orc_step(&p, k + 1, f, g, T)) return 1;
        ops[k] = g_ops;
    }
    std::printf("%llu %llu %ld\n", ops[0], ops[1], N);
    delete[] rho; delete[] u; delete[] T; delete[] f; delete[] g;
    return 0;
}
