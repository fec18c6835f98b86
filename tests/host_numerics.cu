// Host driver for tests/test_host_numerics.py: applies the library's
// error-free FP32 arithmetic (two_sum, the double-float type) and the SPD 3x3
// block inverse of the multigrid smoother to inputs read from stdin, and
// prints the results as hexadecimal floats for exact checking in Python.
//   ts a b                -> s e            (a, b floats)
//   add ahi alo bhi blo   -> hi lo          (double-float sum)
//   mul ahi alo bhi blo   -> hi lo          (double-float product)
//   acc n x_1 .. x_n      -> hi lo          (doubles accumulated with +=)
//   inv a_0 .. a_8        -> o_0 .. o_8     (spd_inv3 of the row-major 3x3)
#include <cstdio>
#include <cstring>
#include "../paper_2511_04025_b300/csrc/common.cuh"
#include "../paper_2511_04025_b300/csrc/mg.cuh"

using namespace shl;

int main() {
    char op[16];
    while (std::scanf("%15s", op) == 1) {
        if (!std::strcmp(op, "ts")) {
            double a, b;
            if (std::scanf("%la %la", &a, &b) != 2) return 2;
            const float2 r = two_sum((float)a, (float)b);
            std::printf("%a %a\n", (double)r.x, (double)r.y);
        } else if (!std::strcmp(op, "add") || !std::strcmp(op, "mul")) {
            double v[4];
            if (std::scanf("%la %la %la %la", v, v + 1, v + 2, v + 3) != 4) return 2;
            const dfloat a((float)v[0], (float)v[1]), b((float)v[2], (float)v[3]);
            const dfloat r = op[0] == 'a' ? a + b : a * b;
            std::printf("%a %a\n", (double)r.hi, (double)r.lo);
        } else if (!std::strcmp(op, "acc")) {
            int n;
            if (std::scanf("%d", &n) != 1) return 2;
            dfloat s(0.0f, 0.0f);
            for (int i = 0; i < n; ++i) {
                double x;
                if (std::scanf("%la", &x) != 1) return 2;
                s += dfloat(x);
            }
            std::printf("%a %a\n", (double)s.hi, (double)s.lo);
        } else if (!std::strcmp(op, "inv")) {
            double a[9], o[9];
            for (int m = 0; m < 9; ++m)
                if (std::scanf("%la", a + m) != 1) return 2;
            spd_inv3(a, o);
            for (int m = 0; m < 9; ++m) std::printf("%a%c", o[m], m == 8 ? '\n' : ' ');
        } else {
            return 3;
        }
    }
    return 0;
}
