// lbfe_analysis.cu -- host-side droplet analysis shared by the observables
// entry points (lbfe_observables and lbfe_observables_noalloc).
//
// Input: the per-plane integer sums the observables kernel writes, six arrays
// of Lx entries over the droplet cells (rho_A > rho_B) of each x-plane:
//   A(x) = #cells, sum y, sum z, sum y^2, sum z^2, sum y z.
// Readings (the paper names the quantities in Secs. 1 and 3 without printing
// their formulas):
//   * x is periodic: the droplet axis is unwrapped from the first occupied
//     plane after the longest circular run of empty planes; L_p = Lx minus
//     that run's length;
//   * D = (a - b)/(a + b) with a, b = sqrt(5 mu / V) from the largest and
//     smallest eigenvalues mu of the second-moment tensor about the centroid
//     (uniform ellipsoid); theta is the major axis' angle from +x in the x-z
//     plane, in (-90, 90] degrees;
//   * necks: interior non-empty local minima of the plateau-compressed A(x)
//     below half the smaller of the adjacent maxima; fragments: occupied
//     x-runs holding >= 1% of the volume; broken = fragments >= 2.
#include <cmath>
#include <cstring>
#include <vector>

#include "lbfe_internal.cuh"

namespace lbfe {

namespace {

int wrap_host(int a, int L) { return ((a % L) + L) % L; }

// Longest empty circular run, unwrapped origin, necks and fragments of A(x).
void analyse_profile(const std::vector<long long> &A, int &Lp, int &start, int &necks, int &frags) {
    const int Lx = (int)A.size();
    long long V = 0;
    for (long long a : A) V += a;
    Lp = start = necks = frags = 0;
    if (V == 0) return;
    int gap = 0, gap_end = 0;
    for (int x = 0; x < Lx; ++x) {
        if (A[x] != 0 || A[wrap_host(x - 1, Lx)] == 0) continue;  // empty run starts at x
        int len = 0;
        while (len < Lx && A[wrap_host(x + len, Lx)] == 0) ++len;
        if (len > gap) { gap = len; gap_end = x + len; }
    }
    start = gap > 0 ? wrap_host(gap_end, Lx) : 0;
    Lp = Lx - gap;
    std::vector<long long> seq(Lp);
    for (int q = 0; q < Lp; ++q) seq[q] = A[wrap_host(start + q, Lx)];
    for (int q = 0; q < Lp;) {
        if (seq[q] == 0) { ++q; continue; }
        long long vol = 0;
        while (q < Lp && seq[q] != 0) vol += seq[q++];
        if (100 * vol >= V) ++frags;
    }
    // plateau-compressed profile framed by empty planes
    std::vector<long long> c{0};
    for (long long v : seq)
        if (v != c.back()) c.push_back(v);
    if (c.back() != 0) c.push_back(0);
    long long prev_max = -1, dip = 0;
    bool have_dip = false;
    for (size_t q = 1; q + 1 < c.size(); ++q) {
        if (c[q] > c[q - 1] && c[q] > c[q + 1]) {
            if (have_dip && prev_max >= 0 && dip > 0 && 2 * dip < std::min(prev_max, c[q])) ++necks;
            prev_max = c[q];
            have_dip = false;
        } else if (c[q] < c[q - 1] && c[q] < c[q + 1]) {
            dip = c[q];
            have_dip = true;
        }
    }
}

}  // namespace

// Eigen-decomposition of a symmetric 3x3 matrix (xx, yy, zz, xy, xz, yz) by
// cyclic Jacobi rotations; eigenvectors are the columns of V.
void sym_eig3(const double M[6], double ev[3], double V[3][3]) {
    double A[3][3] = {{M[0], M[3], M[4]}, {M[3], M[1], M[5]}, {M[4], M[5], M[2]}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = std::fabs(A[0][1]) + std::fabs(A[0][2]) + std::fabs(A[1][2]);
        if (off == 0.0) break;
        for (int pp = 0; pp < 2; ++pp)
            for (int qq = pp + 1; qq < 3; ++qq) {
                if (A[pp][qq] == 0.0) continue;
                const double theta = 0.5 * std::atan2(2.0 * A[pp][qq], A[qq][qq] - A[pp][pp]);
                const double c = std::cos(theta), s = std::sin(theta);
                // rotation in the (pp, qq) plane that zeroes A[pp][qq]
                for (int k = 0; k < 3; ++k) {
                    const double akp = A[k][pp], akq = A[k][qq];
                    A[k][pp] = c * akp - s * akq;
                    A[k][qq] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double apk = A[pp][k], aqk = A[qq][k];
                    A[pp][k] = c * apk - s * aqk;
                    A[qq][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][pp], vkq = V[k][qq];
                    V[k][pp] = c * vkp - s * vkq;
                    V[k][qq] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 3; ++i) ev[i] = A[i][i];
}

void droplet_from_profile(const unsigned long long *prof, int Lx, double R, lbfe_obs *out) {
    std::vector<long long> A(Lx);
    for (int x = 0; x < Lx; ++x) A[x] = (long long)prof[x];
    int Lp, start, necks, frags;
    analyse_profile(A, Lp, start, necks, frags);
    out->Lp = Lp;
    out->Lp_over_2R = R > 0 ? Lp / (2.0 * R) : 0.0;
    out->necks = necks;
    out->fragments = frags;
    out->broken = frags >= 2;
    // moments with the unwrapped x' = (x - start) mod Lx
    double V = 0, sx = 0, sy = 0, sz = 0, sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
    for (int x = 0; x < Lx; ++x) {
        const double xp = (double)wrap_host(x - start, Lx);
        const double a = (double)prof[x];
        V += a;
        sx += xp * a;
        sxx += xp * xp * a;
        sy += (double)prof[Lx + x];
        sz += (double)prof[2 * Lx + x];
        syy += (double)prof[3 * Lx + x];
        szz += (double)prof[4 * Lx + x];
        syz += (double)prof[5 * Lx + x];
        sxy += xp * (double)prof[Lx + x];
        sxz += xp * (double)prof[2 * Lx + x];
    }
    out->volume = V;
    if (V > 0) {
        const double cx = sx / V, cy = sy / V, cz = sz / V;
        out->centroid[0] = std::fmod(cx + start, (double)Lx);
        out->centroid[1] = cy;
        out->centroid[2] = cz;
        double *M = out->M;
        M[0] = sxx - V * cx * cx; M[1] = syy - V * cy * cy; M[2] = szz - V * cz * cz;
        M[3] = sxy - V * cx * cy; M[4] = sxz - V * cx * cz; M[5] = syz - V * cy * cz;
        double ev[3], Vec[3][3];
        sym_eig3(M, ev, Vec);
        int imax = 0, imin = 0;
        for (int q = 1; q < 3; ++q) {
            if (ev[q] > ev[imax]) imax = q;
            if (ev[q] < ev[imin]) imin = q;
        }
        const double a = std::sqrt(5.0 * std::fmax(ev[imax], 0.0) / V);
        const double b = std::sqrt(5.0 * std::fmax(ev[imin], 0.0) / V);
        out->D = (a + b) > 0 ? (a - b) / (a + b) : 0.0;
        double th = std::atan2(Vec[2][imax], Vec[0][imax]) * 180.0 / M_PI;
        if (th <= -90.0) th += 180.0;
        if (th > 90.0) th -= 180.0;
        out->theta_deg = th;
    }
}

}  // namespace lbfe
