// Warp-level helpers of the flux kernels (first-order flux.cu, second-order second_order.cu): the
// lanes of a warp are split into groups of kGroup = 8, one cell per group, 4 cells per warp; each
// lane sums its points and the group's lane sums are combined by a compensated reduce-scatter.
#pragma once

namespace kitrt_flux {

constexpr unsigned kFull = 0xffffffffu;

// Slots of a reduce-scatter of n sums: the next power of two >= n, and its log2.
template <int n>
struct Slots {
    static constexpr int S = n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32;
    static constexpr int H = S == 1 ? 0 : S == 2 ? 1 : S == 4 ? 2 : S == 8 ? 3 : S == 16 ? 4 : 5;
};

constexpr int kGroup = 8;
constexpr int kCellsPerWarp = 32 / kGroup;
constexpr int kGroupLog = 3;

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Compensated reduce-scatter of n per-lane sums over a group of G = 2^kGroupLog lanes. Halving
// levels with offsets G/2, G/4, ... (at most log2 G of them) leave each lane K = S >> H of the
// padded S slots; the remaining levels are compensated butterflies between lanes holding the same
// slots. Lane gl of the group ends with slots base .. base + K - 1, base = (gl >> (log2 G - H)) K,
// values rs[k] + re[k]; it returns whether it is the unique holder of them.
template <int n>
struct GroupRS {
    static constexpr int S = Slots<n>::S;
    static constexpr int H = Slots<n>::H < kGroupLog ? Slots<n>::H : kGroupLog;
    static constexpr int K = S >> H;
};

template <int n>
__device__ __forceinline__ bool group_reduce_scatter(const float (&F)[n], int gl,
                                                     float (&rs)[GroupRS<n>::K],
                                                     float (&re)[GroupRS<n>::K], int &base)
{
    constexpr int S = GroupRS<n>::S, H = GroupRS<n>::H, K = GroupRS<n>::K;
    float sv[S], ev[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
        sv[k] = k < n ? F[k < n ? k : 0] : 0.0f;
        ev[k] = 0.0f;
    }
#pragma unroll
    for (int lvl = 0; lvl < H; ++lvl) {
        const int o = (1 << (kGroupLog - 1)) >> lvl;
        const int half = S >> (lvl + 1);
        const bool upper = (gl & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const float ks = upper ? sv[k + half] : sv[k], ke = upper ? ev[k + half] : ev[k];
            const float xs = upper ? sv[k] : sv[k + half], xe = upper ? ev[k] : ev[k + half];
            const float ps = __shfl_xor_sync(kFull, xs, o), pe = __shfl_xor_sync(kFull, xe, o);
            float t, e;
            two_sum(ks, ps, t, e);
            sv[k] = t;
            ev[k] = ke + pe + e;
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float s0 = sv[k], e0 = ev[k];
#pragma unroll
        for (int o = (1 << (kGroupLog - 1)) >> H; o > 0; o >>= 1) {
            const float so = __shfl_xor_sync(kFull, s0, o), eo = __shfl_xor_sync(kFull, e0, o);
            float t, e;
            two_sum(s0, so, t, e);
            s0 = t;
            e0 = e0 + eo + e;
        }
        rs[k] = s0;
        re[k] = e0;
    }
    base = (gl >> (kGroupLog - H)) * K;
    return (gl & ((1 << (kGroupLog - H)) - 1)) == 0;
}

}  // namespace kitrt_flux
