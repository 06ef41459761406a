// FFT plan of one control point class (N, r): how the template is cut into
// blocks and which 2-D FFT size correlates each block with its search window.
//
// Sec. III-G computes the SSD surface of Eq. 3 through FFT correlation
// (Eq. 8-9).  The correlation is linear in the template, so the template may
// be cut into nb_y x nb_x blocks: each block of size b_y x b_x is correlated
// with its own (b_y + 2r) x (b_x + 2r) window and the cross-spectra of all
// blocks and channels are summed before one inverse FFT.  A P_y x P_x FFT
// with P >= b + 2r gives every lag in [-r, r] without circular wrap.  Every
// FFT length is a product P = A * B of two register radices, A, B in
// {2,3,4,5,6,8,9,10,12,15,16} (B = 1 allowed): two shared-memory passes per
// axis.  The plan depends only on (N, r, m) and the kernel variant's plane
// bound, so a CP's result never depends on its batch.  The search is exact
// integer arithmetic: host and device agree.
#pragma once

#include <cstdint>

namespace cfog {

constexpr int kMaxFft = 256;           // longest supported FFT side
constexpr int kMaxPlaneElems = 16384;  // largest P_y * P_x of any kernel variant
constexpr int kNbMax = 4;              // blocks per axis searched
constexpr int kPTries = 4;             // FFT lengths tried per axis

struct FftDim {
    int nb;   // number of template blocks along this axis
    int bs;   // block size ceil(N / nb); the last block may be shorter
    int P;    // FFT length, even
    int A;    // stage-1 radix (stride B)
    int B;    // stage-2 radix (contiguous); 1 = single stage
};

struct MatchPlan {
    FftDim y, x;
};

constexpr bool is_radix(int R) {
    return R == 2 || R == 3 || R == 4 || R == 5 || R == 6 || R == 8 || R == 9 || R == 10 ||
           R == 12 || R == 15 || R == 16;
}

// Split of every even length P <= kMaxFft into A * B (register radices, B may
// be 1), as balanced as possible (ties: smaller A), and the smallest
// splittable length >= P.  Built at compile time; the host and the device
// read the same table.
struct SmoothTable {
    unsigned char A[kMaxFft + 1];
    unsigned char B[kMaxFft + 1];
    unsigned short next[kMaxFft + 2];   // 0: none up to kMaxFft
    constexpr SmoothTable() : A(), B(), next() {
        for (int P = 0; P <= kMaxFft; ++P) {
            A[P] = 0;
            B[P] = 0;
            if (P < 2 || (P & 1)) continue;
            int bestA = 0, bestB = 0, bestd = 1 << 30;
            for (int a = 2; a <= 16; ++a) {
                if (!is_radix(a) || P % a) continue;
                const int b = P / a;
                if (b != 1 && !is_radix(b)) continue;
                const int d = a > b ? a - b : b - a;
                if (d < bestd) {
                    bestd = d;
                    bestA = a;
                    bestB = b;
                }
            }
            A[P] = (unsigned char)bestA;
            B[P] = (unsigned char)bestB;
        }
        next[kMaxFft + 1] = 0;
        for (int P = kMaxFft; P >= 0; --P) next[P] = A[P] ? (unsigned short)P : next[P + 1];
    }
};

constexpr SmoothTable kSmoothHost{};
static __constant__ const SmoothTable kSmoothDev = SmoothTable{};

__host__ __device__ inline const SmoothTable &smooth_table() {
#ifdef __CUDA_ARCH__
    return kSmoothDev;
#else
    return kSmoothHost;
#endif
}

// Split an even P into A * B; returns false when no split exists.
__host__ __device__ inline bool fft_split(int P, int *A, int *B) {
    const SmoothTable &t = smooth_table();
    if (P < 0 || P > kMaxFft || !t.A[P]) return false;
    *A = t.A[P];
    *B = t.B[P];
    return true;
}

__host__ __device__ inline int ceil_log2(int v) {
    int c = 0;
    while ((1 << c) < v) ++c;
    return c;
}

// Integer cost of one length-P pass over a plane: each stage is a
// shared-memory round trip (100) plus arithmetic ~ log2 of its radix.
__host__ __device__ inline int fft_len_cost(int A, int B) {
    return 100 + 12 * ceil_log2(A) + (B > 1 ? 100 + 12 * ceil_log2(B) : 0);
}

// Best (Py, Px) for one block split (nby, nbx) with P_y * P_x <= maxe (the
// kernel variant's shared-memory plane); returns the cost (or -1 when no
// size fits) and fills *out.  Scan order: Py ascending, then Px ascending;
// a later candidate wins only with a strictly smaller cost.
__host__ __device__ inline long long plan_for_split(int N, int r, int m, int nby, int nbx,
                                                    int maxe, MatchPlan *out) {
    const int bsy = (N + nby - 1) / nby, bsx = (N + nbx - 1) / nbx;
    if ((nby - 1) * bsy >= N || (nbx - 1) * bsx >= N) return -1;
    const int needy = bsy + 2 * r, needx = bsx + 2 * r;
    long long best = -1;
    if (needy > kMaxFft || needx > kMaxFft) return -1;
    const SmoothTable &t = smooth_table();
    int tried_y = 0;
    for (int Py = t.next[needy]; Py != 0 && tried_y < kPTries; Py = t.next[Py + 1]) {
        const int Ay = t.A[Py], By = t.B[Py];
        ++tried_y;
        int tried_x = 0;
        for (int Px = t.next[needx]; Px != 0 && tried_x < kPTries; Px = t.next[Px + 1]) {
            const int Ax = t.A[Px], Bx = t.B[Px];
            ++tried_x;
            if (Py * Px > maxe) continue;
            // the row box sums of the ||D||^2 window (W x L floats) use the plane
            // as scratch before the FFTs
            if (2LL * Py * (Px + 1) < (long long)(N + 2 * r) * (2 * r + 1)) continue;
            const long long per = (long long)Py * Px * (fft_len_cost(Ay, By) + fft_len_cost(Ax, Bx));
            const long long cost = per * (long long)(nby * nbx * m + 1);
            if (best < 0 || cost < best) {
                best = cost;
                out->y = FftDim{nby, bsy, Py, Ay, By};
                out->x = FftDim{nbx, bsx, Px, Ax, Bx};
            }
        }
    }
    return best;
}

// A plan named by a code: bits 4..7 the split index l (nby = l / kNbMax + 1,
// nbx = l % kNbMax + 1), bits 2..3 and 0..1 which of the first kPTries
// splittable lengths >= b + 2r the y and x axes take.  Returns the cost of
// plan_for_split's model (or -1 when the code names no feasible plan) and
// fills *out.  The autotuner times codes and records the fastest per class.
constexpr int kPlanCodes = kNbMax * kNbMax * kPTries * kPTries;

__host__ __device__ inline long long plan_for_code(int N, int r, int m, int code, int maxe,
                                                   MatchPlan *out) {
    if (code < 0 || code >= kPlanCodes) return -1;
    const int l = code >> 4, ty = (code >> 2) & 3, tx = code & 3;
    const int nby = l / kNbMax + 1, nbx = l % kNbMax + 1;
    const int bsy = (N + nby - 1) / nby, bsx = (N + nbx - 1) / nbx;
    if ((nby - 1) * bsy >= N || (nbx - 1) * bsx >= N) return -1;
    const int needy = bsy + 2 * r, needx = bsx + 2 * r;
    if (needy > kMaxFft || needx > kMaxFft) return -1;
    const SmoothTable &t = smooth_table();
    int Py = t.next[needy];
    for (int i = 0; i < ty && Py != 0; ++i) Py = t.next[Py + 1];
    int Px = t.next[needx];
    for (int i = 0; i < tx && Px != 0; ++i) Px = t.next[Px + 1];
    if (Py == 0 || Px == 0 || Py * Px > maxe) return -1;
    if (2LL * Py * (Px + 1) < (long long)(N + 2 * r) * (2 * r + 1)) return -1;
    const int Ay = t.A[Py], By = t.B[Py], Ax = t.A[Px], Bx = t.B[Px];
    const long long per = (long long)Py * Px * (fft_len_cost(Ay, By) + fft_len_cost(Ax, Bx));
    out->y = FftDim{nby, bsy, Py, Ay, By};
    out->x = FftDim{nbx, bsx, Px, Ax, Bx};
    return per * (long long)(nby * nbx * m + 1);
}

// Split index l in [0, kNbMax^2): nby = l / kNbMax + 1, nbx = l % kNbMax + 1.
// The plan is the split with the smallest cost, ties to the smaller l.
__host__ inline bool make_plan_host(int N, int r, int m, int maxe, MatchPlan *out) {
    long long best = -1;
    for (int l = 0; l < kNbMax * kNbMax; ++l) {
        MatchPlan p;
        const long long c = plan_for_split(N, r, m, l / kNbMax + 1, l % kNbMax + 1, maxe, &p);
        if (c >= 0 && (best < 0 || c < best)) {
            best = c;
            *out = p;
        }
    }
    return best >= 0;
}

// Row pitch of the shared-memory plane: odd, so that threads walking down a
// column of complex values hit distinct banks.
__host__ __device__ inline int plane_ld(const MatchPlan &p) { return p.x.P + 1; }

// Dynamic shared memory of the FP32 FFT match kernel for a plan and radius r:
// the complex plane, the twiddles of both axes, the accumulator position
// table and the (2r+1)^2 box sums.
__host__ __device__ inline int plan_smem_bytes(const MatchPlan &p, int r) {
    return p.y.P * plane_ld(p) * 8 + (p.y.P + p.x.P) * 8 + p.y.P * (p.x.P / 2 + 1) * 4 +
           (2 * r + 1) * (2 * r + 1) * 4;
}

}  // namespace cfog
