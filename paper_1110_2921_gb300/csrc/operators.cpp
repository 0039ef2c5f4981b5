// Host-side FP64 construction of the translation operators of the periodic FMM.
//
// Expansions are in solid harmonics (Section 3.1, Eqs. fmm3dm and fmm3dl).  We use the
// regular / irregular solid harmonics defined by the recurrences
//   Y_0^0 = 1,  Y_n^n = -(x + i y)/(2n) Y_{n-1}^{n-1},
//   Y_n^m = ((2n-1) z Y_{n-1}^m - r^2 Y_{n-2}^m) / ((n+m)(n-m)),
//   T_0^0 = 1/r, T_n^n = -(2n-1)(x + i y)/r^2 T_{n-1}^{n-1},
//   T_n^m = ((2n-1) z T_{n-1}^m - ((n-1)^2 - m^2) T_{n-2}^m) / r^2,
// with A_n^{-m} = (-1)^m conj(A_n^m).  They satisfy 1/|x-y| = sum conj(Y_n^m(y)) T_n^m(x)
// (|y| < |x|), the addition theorems Y(a+b) = sum Y_k^l(a) Y_{n-k}^{m-l}(b) and
// T(x-y) = sum conj(Y_k^l(y)) T_{n+k}^{m+l}(x), and d/dz Y_n^m = Y_{n-1}^m,
// (d/dx + i d/dy) Y_n^m = Y_{n-1}^{m+1}, (d/dx - i d/dy) Y_n^m = -Y_{n-1}^{m-1}.
//
// Coefficients are stored "balanced" so that every value and every operator entry is
// O(1) for any level (needed by the BF16/TF32 tensor-core M2L):
//   multipole  Mh_n^m = s_nm / w^n * sum_j q_j Y_n^m(x_j - z)
//   local      potential(x) = (1/w) sum_{k,l} conj(Y_k^l((x - z)/w)) s_kl Fh_k^l
// with s_nm = sqrt((n+m)! (n-m)!) and w the cell width.  Only m >= 0 is stored, packed as
// [n^2] = Re A_n^0, [n^2 + 2m - 1] = Re A_n^m, [n^2 + 2m] = Im A_n^m; every operator is a
// real (p+1)^2 x (p+1)^2 matrix on this packing.
#include "vfmm_internal.h"

#include <cmath>
#include <complex>
#include <vector>

namespace vfmm {
namespace ops {

typedef std::complex<double> cd;

struct Harm {
    int p;
    std::vector<cd> a;  // (n, m >= 0) at n*(p+1)+m
    cd get(int n, int m) const
    {
        if (n < 0 || n > p) return cd(0.0, 0.0);
        int am = m < 0 ? -m : m;
        if (am > n) return cd(0.0, 0.0);
        cd v = a[n * (p + 1) + am];
        if (m >= 0) return v;
        return (am & 1) ? -std::conj(v) : std::conj(v);
    }
};

static Harm regular(const double v[3], int p)
{
    Harm U;
    U.p = p;
    U.a.assign((p + 1) * (p + 1), cd(0.0, 0.0));
    double x = v[0], y = v[1], z = v[2], r2 = x * x + y * y + z * z;
    U.a[0] = 1.0;
    for (int n = 1; n <= p; ++n) U.a[n * (p + 1) + n] = -cd(x, y) / (2.0 * n) * U.a[(n - 1) * (p + 1) + n - 1];
    for (int m = 0; m <= p; ++m)
        for (int n = m + 1; n <= p; ++n) {
            cd prev2 = (n - 2 >= m) ? U.a[(n - 2) * (p + 1) + m] : cd(0.0, 0.0);
            U.a[n * (p + 1) + m] = ((2.0 * n - 1.0) * z * U.a[(n - 1) * (p + 1) + m] - r2 * prev2) /
                                   double((n + m) * (n - m));
        }
    return U;
}

static Harm irregular(const double v[3], int p)
{
    Harm T;
    T.p = p;
    T.a.assign((p + 1) * (p + 1), cd(0.0, 0.0));
    double x = v[0], y = v[1], z = v[2], r2 = x * x + y * y + z * z;
    T.a[0] = 1.0 / std::sqrt(r2);
    for (int n = 1; n <= p; ++n)
        T.a[n * (p + 1) + n] = -(2.0 * n - 1.0) * cd(x, y) / r2 * T.a[(n - 1) * (p + 1) + n - 1];
    for (int m = 0; m <= p; ++m)
        for (int n = m + 1; n <= p; ++n) {
            cd prev2 = (n - 2 >= m) ? T.a[(n - 2) * (p + 1) + m] : cd(0.0, 0.0);
            T.a[n * (p + 1) + m] = ((2.0 * n - 1.0) * z * T.a[(n - 1) * (p + 1) + m] -
                                    double((n - 1) * (n - 1) - m * m) * prev2) / r2;
        }
    return T;
}

double sfac(int n, int m)
{
    double a = 1.0;
    for (int k = 2; k <= n + m; ++k) a *= k;
    double b = 1.0;
    for (int k = 2; k <= n - m; ++k) b *= k;
    return std::sqrt(a * b);
}

static inline int pidx(int n, int m, int part) { return m == 0 ? n * n : n * n + 2 * m - 1 + part; }

// Decode packed index j into (n, m, part, v) with v = 1 (real part) or i (imaginary part).
static void decode(int j, int &n, int &m, cd &v)
{
    n = (int)std::floor(std::sqrt((double)j));
    while ((n + 1) * (n + 1) <= j) ++n;
    while (n * n > j) --n;
    int r = j - n * n;
    if (r == 0) {
        m = 0;
        v = cd(1.0, 0.0);
    } else {
        m = (r + 1) / 2;
        v = (r & 1) ? cd(1.0, 0.0) : cd(0.0, 1.0);
    }
}

static void put(std::vector<double> &A, int nc, int row_n, int row_m, int col, cd val)
{
    A[(size_t)pidx(row_n, row_m, 0) * nc + col] += val.real();
    if (row_m > 0) A[(size_t)pidx(row_n, row_m, 1) * nc + col] += val.imag();
}

// M2L: Fh_k^l = (-1)^k sum_{n,m} conj(Mh_n^m) T_{n+k}^{m+l}(t) / (s_kl s_nm),
// t = (target centre - source centre) / w.  (Derived from the irregular addition theorem.)
std::vector<double> m2l_hat(const double t[3], int p)
{
    int nc = (p + 1) * (p + 1);
    std::vector<double> A((size_t)nc * nc, 0.0);
    Harm T = irregular(t, 2 * p);
    for (int j = 0; j < nc; ++j) {
        int n, m;
        cd v;
        decode(j, n, m, v);
        double snm = sfac(n, m);
        for (int k = 0; k <= p; ++k)
            for (int l = 0; l <= k; ++l) {
                cd val = std::conj(v) * T.get(n + k, m + l);
                if (m > 0) val += ((m & 1) ? -1.0 : 1.0) * v * T.get(n + k, l - m);
                val *= ((k & 1) ? -1.0 : 1.0) / (sfac(k, l) * snm);
                put(A, nc, k, l, j, val);
            }
    }
    return A;
}

// M2M from a child (width w) to its parent (width ratio*w):
// Mh'_n^m = s_nm sum_{k,l} Y_{n-k}^{m-l}(e) Mh_k^l ratio^-k / s_kl,
// e = (child centre - parent centre) / (parent width).
std::vector<double> m2m_hat(const double e[3], double ratio, int p)
{
    int nc = (p + 1) * (p + 1);
    std::vector<double> A((size_t)nc * nc, 0.0);
    Harm U = regular(e, p);
    for (int j = 0; j < nc; ++j) {
        int k, l;
        cd v;
        decode(j, k, l, v);
        double f = std::pow(ratio, -k) / sfac(k, l);
        for (int n = k; n <= p; ++n)
            for (int m = 0; m <= n; ++m) {
                cd val = U.get(n - k, m - l) * v;
                if (l > 0) val += U.get(n - k, m + l) * ((l & 1) ? -1.0 : 1.0) * std::conj(v);
                val *= sfac(n, m) * f;
                put(A, nc, n, m, j, val);
            }
    }
    return A;
}

// L2L from a parent (width 2w) to a child (width w):
// Fh'_a^b = (1/s_ab) sum_{k,l} conj(Y_{k-a}^{l-b}(e)) Fh_k^l s_kl 2^-(k+1),
// e = (child centre - parent centre) / (child width).
std::vector<double> l2l_hat(const double e[3], int p)
{
    int nc = (p + 1) * (p + 1);
    std::vector<double> A((size_t)nc * nc, 0.0);
    Harm U = regular(e, p);
    for (int j = 0; j < nc; ++j) {
        int k, l;
        cd v;
        decode(j, k, l, v);
        double f = sfac(k, l) * std::pow(2.0, -(k + 1));
        for (int a = 0; a <= k; ++a)
            for (int b = 0; b <= a; ++b) {
                cd val = std::conj(U.get(k - a, l - b)) * v;
                if (l > 0) val += std::conj(U.get(k - a, -l - b)) * ((l & 1) ? -1.0 : 1.0) * std::conj(v);
                val *= f / sfac(a, b);
                put(A, nc, a, b, j, val);
            }
    }
    return A;
}

static std::vector<double> matmul(const std::vector<double> &A, const std::vector<double> &B, int n)
{
    std::vector<double> C((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            double a = A[(size_t)i * n + k];
            if (a == 0.0) continue;
            for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += a * B[(size_t)k * n + j];
        }
    return C;
}

// Periodic lattice operator: root multipole (hat, w = L) -> root local (hat, w = L) for the
// image boxes outside the central 3^3 and inside the cube of 3^(S+1) boxes per side.
// Super-level l treats the 3^l L block around the root as one cell: its interaction list is
// the 702 blocks at offsets i, i in {-4..4}^3 minus {-1..1}^3 (children of the 3^(l+1) L
// parent's 27 neighbours minus its own 27); the next super-cell's multipole is the M2M sum of
// 27 copies at offsets c in {-1,0,1}^3.  All cells share one centre, so no L2L is needed; the
// local of super-level l is rescaled to root units by 3^(-l(k+1)).
std::vector<double> lattice_operator(int p, int S)
{
    int nc = (p + 1) * (p + 1);
    std::vector<double> Op((size_t)nc * nc, 0.0);
    if (S <= 0) return Op;
    std::vector<double> Asum((size_t)nc * nc, 0.0), Bsum((size_t)nc * nc, 0.0);
    for (int ix = -4; ix <= 4; ++ix)
        for (int iy = -4; iy <= 4; ++iy)
            for (int iz = -4; iz <= 4; ++iz) {
                if (std::abs(ix) <= 1 && std::abs(iy) <= 1 && std::abs(iz) <= 1) continue;
                double t[3] = {-(double)ix, -(double)iy, -(double)iz};
                std::vector<double> A = m2l_hat(t, p);
                for (size_t q = 0; q < A.size(); ++q) Asum[q] += A[q];
            }
    for (int cx = -1; cx <= 1; ++cx)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cz = -1; cz <= 1; ++cz) {
                double e[3] = {cx / 3.0, cy / 3.0, cz / 3.0};
                std::vector<double> B = m2m_hat(e, 3.0, p);
                for (size_t q = 0; q < B.size(); ++q) Bsum[q] += B[q];
            }
    std::vector<double> chain((size_t)nc * nc, 0.0);  // B^l, starts at identity
    for (int i = 0; i < nc; ++i) chain[(size_t)i * nc + i] = 1.0;
    for (int l = 0; l < S; ++l) {
        std::vector<double> AB = matmul(Asum, chain, nc);
        for (int k = 0; k <= p; ++k) {
            double sc = std::pow(3.0, -(double)l * (k + 1));
            for (int row = k * k; row < (k + 1) * (k + 1); ++row)
                for (int c = 0; c < nc; ++c) Op[(size_t)row * nc + c] += sc * AB[(size_t)row * nc + c];
        }
        chain = matmul(Bsum, chain, nc);
    }
    return Op;
}

}  // namespace ops
}  // namespace vfmm
