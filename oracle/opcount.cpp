/*
 * opcount.cpp -- the oracle compiled with every `double` replaced by a type
 * that counts the floating-point operations performed on it.
 *
 * TEST INFRASTRUCTURE, like sensei_oracle.c itself: it exists to give the
 * exact number of arithmetic operations the method (as the oracle states it,
 * Sec. 2-3) performs per cell, the algorithmic operation count against which
 * a kernel's throughput is measured.  Only the tests and the bench's
 * constants (checked by a test) use it.
 *
 * The counting type holds one double and nothing else, so arrays, structs
 * and the by-value arguments of the exported functions keep the layout and
 * calling convention of double (a trivially copyable one-member aggregate of
 * a double travels in a floating-point register on the x86-64 and AArch64
 * calling conventions): the same ctypes bindings drive either build.
 *
 * Counted: additions and subtractions, multiplications, divisions, square
 * roots, comparisons, absolute values and min/max, negations.  The values are
 * computed in plain double exactly as in the C build (-ffp-contract=off).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

struct ora_opcounts {
    unsigned long long add, mul, div, sqrt, cmp, abs, neg;
};
static ora_opcounts g_ops;

struct ora_counted {
    double v;
    ora_counted() = default;
    ora_counted(double x) : v(x) {}
    explicit operator long() const { return (long)v; }
    explicit operator int() const { return (int)v; }
};

static inline ora_counted operator+(ora_counted a, ora_counted b) { ++g_ops.add; return a.v + b.v; }
static inline ora_counted operator-(ora_counted a, ora_counted b) { ++g_ops.add; return a.v - b.v; }
static inline ora_counted operator*(ora_counted a, ora_counted b) { ++g_ops.mul; return a.v * b.v; }
static inline ora_counted operator/(ora_counted a, ora_counted b) { ++g_ops.div; return a.v / b.v; }
static inline ora_counted operator-(ora_counted a) { ++g_ops.neg; return -a.v; }
static inline ora_counted operator+(ora_counted a) { return a; }
static inline ora_counted &operator+=(ora_counted &a, ora_counted b) { return a = a + b; }
static inline ora_counted &operator-=(ora_counted &a, ora_counted b) { return a = a - b; }
static inline ora_counted &operator*=(ora_counted &a, ora_counted b) { return a = a * b; }
static inline ora_counted &operator/=(ora_counted &a, ora_counted b) { return a = a / b; }
static inline bool operator<(ora_counted a, ora_counted b) { ++g_ops.cmp; return a.v < b.v; }
static inline bool operator>(ora_counted a, ora_counted b) { ++g_ops.cmp; return a.v > b.v; }
static inline bool operator<=(ora_counted a, ora_counted b) { ++g_ops.cmp; return a.v <= b.v; }
static inline bool operator>=(ora_counted a, ora_counted b) { ++g_ops.cmp; return a.v >= b.v; }
static inline bool operator==(ora_counted a, ora_counted b) { ++g_ops.cmp; return a.v == b.v; }
static inline bool operator!=(ora_counted a, ora_counted b) { ++g_ops.cmp; return a.v != b.v; }
static inline ora_counted sqrt(ora_counted a) { ++g_ops.sqrt; return ::sqrt(a.v); }
static inline ora_counted fabs(ora_counted a) { ++g_ops.abs; return ::fabs(a.v); }
static inline ora_counted fmax(ora_counted a, ora_counted b) { ++g_ops.abs; return ::fmax(a.v, b.v); }
static inline ora_counted fmin(ora_counted a, ora_counted b) { ++g_ops.abs; return ::fmin(a.v, b.v); }

#define double ora_counted
extern "C" {
#include "sensei_oracle.c"
}
#undef double

extern "C" {
void ora_opcount_reset(void) { memset(&g_ops, 0, sizeof(g_ops)); }

/* out[0..6] = additions/subtractions, multiplications, divisions, square
 * roots, comparisons, absolute values and min/max, negations */
void ora_opcount_get(unsigned long long out[7])
{
    out[0] = g_ops.add;
    out[1] = g_ops.mul;
    out[2] = g_ops.div;
    out[3] = g_ops.sqrt;
    out[4] = g_ops.cmp;
    out[5] = g_ops.abs;
    out[6] = g_ops.neg;
}
}
