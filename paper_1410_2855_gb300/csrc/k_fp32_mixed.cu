// FP32 fused path, one launch per sweep for size classes of uneven grid
// sizes (sweep_mixed.cuh): launch plans and launchers.
#include <climits>
#include <cstring>

#include "launch.cuh"
#include "sweep_mixed.cuh"

namespace rtk {

bool mix_supported(int logn) { return logn >= kMixMinLog && logn <= kMixMaxLog; }
int mix_col_tile(int logn) { return mix_col_width(logn); }

namespace {

template <typename K> cudaError_t mix_attr(K k, size_t smem, std::atomic<unsigned long long> &mask)
{
    return ensure_smem(k, smem, mask);
}

// The items of the given classes (all within the supported sides), in order.
cudaError_t make_plan(const MixLaunch *cls, int ncls, bool col, MixPlan *p)
{
    if (ncls <= 0 || ncls > kMixMaxClasses) return cudaErrorInvalidValue;
    std::memset(p, 0, sizeof(*p));
    long long items = 0;
    for (int k = 0; k < ncls; ++k) {
        const MixLaunch &c = cls[k];
        if (!mix_supported(c.logn) || c.nres <= 0) return cudaErrorInvalidValue;
        const long long n2 = 1ll << (2 * c.logn);
        const int per = (int)(n2 / (col ? kMixColPoints : kMixRowPoints));
        p->c[k] = {c.res, c.tw, c.nres, c.logn, (int)items, per};
        items += (long long)c.nres * per;
    }
    if (items > INT_MAX / 2) return cudaErrorInvalidValue;
    p->ncls = ncls;
    p->nitems = (int)items;
    return cudaSuccess;
}

}  // namespace

cudaError_t prepare_mixed32()
{
    static std::atomic<unsigned long long> mc{0}, mr{0};
    cudaError_t e = mix_attr(k_col_mixed, kMixColSmem, mc);
    if (e == cudaSuccess) e = mix_attr(k_row_mixed, kMixRowSmem, mr);
    return e;
}

cudaError_t launch_col_mixed32(const MixLaunch *cls, int ncls, int *err, cudaStream_t s)
{
    MixPlan p;
    cudaError_t e = make_plan(cls, ncls, true, &p);
    if (e != cudaSuccess) return e;
    static std::atomic<unsigned long long> mask{0};
    static std::atomic<int> per_sm{0};
    if ((e = mix_attr(k_col_mixed, kMixColSmem, mask)) != cudaSuccess) return e;
    const int grid = persistent_grid(k_col_mixed, kMixColThreads, kMixColSmem, p.nitems, per_sm);
    k_col_mixed<<<grid, kMixColThreads, kMixColSmem, s>>>(p, err);
    return cudaGetLastError();
}

cudaError_t launch_row_mixed32(const MixLaunch *cls, int ncls, int *err, cudaStream_t s)
{
    MixPlan p;
    cudaError_t e = make_plan(cls, ncls, false, &p);
    if (e != cudaSuccess) return e;
    static std::atomic<unsigned long long> mask{0};
    static std::atomic<int> per_sm{0};
    if ((e = mix_attr(k_row_mixed, kMixRowSmem, mask)) != cudaSuccess) return e;
    const int grid = persistent_grid(k_row_mixed, kMixRowThreads, kMixRowSmem, p.nitems, per_sm);
    k_row_mixed<<<grid, kMixRowThreads, kMixRowSmem, s>>>(p, err);
    return cudaGetLastError();
}

}  // namespace rtk
