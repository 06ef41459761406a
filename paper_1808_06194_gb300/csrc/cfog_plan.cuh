// FFT plan of one control point class (N, r): how the template is cut into
// blocks and which 2-D FFT size correlates each block with its search window.
//
// Sec. III-G computes the SSD surface of Eq. 3 through FFT correlation
// (Eq. 8-9).  The correlation is linear in the template, so the template may
// be cut into nb_y x nb_x blocks: each block of size b_y x b_x is correlated
// with its own (b_y + 2r) x (b_x + 2r) window and the cross-spectra of all
// blocks and channels are summed before one inverse FFT.  A P_y x P_x FFT
// with P >= b + 2r gives every lag in [-r, r] without circular wrap.  The plan
// depends only on (N, r, m), so a CP's result never depends on its batch.
// The search is exact integer arithmetic, so host and device agree bit for bit.
#pragma once

#include <cstdint>

namespace cfog {

constexpr int kMaxFft = 256;          // longest supported FFT side
constexpr int kMaxPlaneElems = 16384; // P_y * P_x bound (plane + half spectrum in smem)
constexpr int kMaxStages = 8;
constexpr int kNbMax = 4;             // blocks per axis searched
constexpr int kPTries = 4;            // smooth FFT lengths tried per axis

struct FftDim {
    int nb;                 // number of template blocks along this axis
    int bs;                 // block size ceil(N / nb); the last block may be shorter
    int P;                  // FFT length (even, 2-3-5 smooth)
    int ns;                 // number of radix stages
    int rad[kMaxStages];    // radices in decimation-in-frequency order
};

struct MatchPlan {
    FftDim y, x;
};

// Factor P into radix-4, -2, -3, -5 stages; 0 if P is odd or not 2-3-5 smooth.
__host__ __device__ inline int fft_factor(int P, int *rad) {
    if (P < 2 || (P & 1)) return 0;
    int n = P, c2 = 0, c3 = 0, c5 = 0, ns = 0;
    while (n % 2 == 0) { n /= 2; ++c2; }
    while (n % 3 == 0) { n /= 3; ++c3; }
    while (n % 5 == 0) { n /= 5; ++c5; }
    if (n != 1) return 0;
    while (c2 >= 2) { rad[ns++] = 4; c2 -= 2; }
    if (c2) rad[ns++] = 2;
    while (c3-- > 0) rad[ns++] = 3;
    while (c5-- > 0) rad[ns++] = 5;
    return ns;
}

// Cost of one length-P pass over a plane, in integer units: each stage is a
// shared-memory round trip (100) plus arithmetic growing with the radix.
__host__ __device__ inline int fft_len_cost(int ns, const int *rad) {
    int c = 0;
    for (int i = 0; i < ns; ++i) c += 100 + 8 * rad[i];
    return c;
}

// Best (Py, Px) for one block split (nby, nbx); returns the cost (or -1 when
// no size fits) and fills *out.  Scan order: Py ascending, then Px ascending;
// a later candidate wins only with a strictly smaller cost.
__host__ __device__ inline long long plan_for_split(int N, int r, int m, int nby, int nbx,
                                                    MatchPlan *out) {
    const int bsy = (N + nby - 1) / nby, bsx = (N + nbx - 1) / nbx;
    if ((nby - 1) * bsy >= N || (nbx - 1) * bsx >= N) return -1;
    const int needy = bsy + 2 * r, needx = bsx + 2 * r;
    long long best = -1;
    int tried_y = 0;
    for (int Py = needy; Py <= kMaxFft && tried_y < kPTries; ++Py) {
        int ry[kMaxStages];
        const int sy = fft_factor(Py, ry);
        if (!sy) continue;
        ++tried_y;
        int tried_x = 0;
        for (int Px = needx; Px <= kMaxFft && tried_x < kPTries; ++Px) {
            int rx[kMaxStages];
            const int sx = fft_factor(Px, rx);
            if (!sx) continue;
            ++tried_x;
            if (Py * Px > kMaxPlaneElems) continue;
            const long long per = (long long)Py * Px * (fft_len_cost(sy, ry) + fft_len_cost(sx, rx));
            const long long cost = per * (long long)(nby * nbx * (m + 1) + 1);
            if (best < 0 || cost < best) {
                best = cost;
                out->y.nb = nby; out->y.bs = bsy; out->y.P = Py; out->y.ns = sy;
                out->x.nb = nbx; out->x.bs = bsx; out->x.P = Px; out->x.ns = sx;
                for (int i = 0; i < sy; ++i) out->y.rad[i] = ry[i];
                for (int i = 0; i < sx; ++i) out->x.rad[i] = rx[i];
            }
        }
    }
    return best;
}

// Split index l in [0, kNbMax^2): nby = l / kNbMax + 1, nbx = l % kNbMax + 1.
// The plan is the split with the smallest cost, ties to the smaller l.
__host__ inline bool make_plan_host(int N, int r, int m, MatchPlan *out) {
    long long best = -1;
    for (int l = 0; l < kNbMax * kNbMax; ++l) {
        MatchPlan p;
        const long long c = plan_for_split(N, r, m, l / kNbMax + 1, l % kNbMax + 1, &p);
        if (c >= 0 && (best < 0 || c < best)) {
            best = c;
            *out = p;
        }
    }
    return best >= 0;
}

// Dynamic shared memory of the FP32 FFT match kernel for a plan.
__host__ __device__ inline int plan_smem_bytes(const MatchPlan &p) {
    const int Py = p.y.P, Px = p.x.P;
    const int plane = Py * Px * 8;
    const int half = Py * (Px / 2 + 1) * 8;
    const int tables = 2 * kMaxFft * 8 + 2 * kMaxFft * 4;
    return plane + half + tables;
}

}  // namespace cfog
