// k_fixed.cuh -- instantiation of the compile-time pass kernels for one half of
// the fixed-plan list (plans.h); each half is its own translation unit so the
// two compile in parallel.
#pragma once

#include "pass_kernels.cuh"
#include "plans.h"
#include "pass_tc.cuh"
#include "pass_tma.cuh"
#include "slab_l2.cuh"

namespace fft3 {

template <int N, int T>
constexpr bool has_slab_l2() { return (N == 1024 || N == 512 || N == 256) && T * kSlabL2Lpt <= 1024; }

template <int N, int T, class Rad>
constexpr const void *slab_l2_ptr()
{
    if constexpr (has_slab_l2<N, T>())
        return (const void *)&k_slab_l2<N, T, Rad, kSlabL2Lpt>;
    else
        return nullptr;
}

template <int N, int T, class Rad, int LPT>
constexpr const void *slab_blk_ptr()
{
    if constexpr (has_slab_l2<N, T>() && T * LPT + 32 <= 1024 &&
                  slab_tma_smem(N, LPT) <= 227 * 1024)
        return (const void *)&k_slab_tma<N, T, Rad, LPT, kSlabTmaBufs>;
    else
        return nullptr;
}

template <int N, int T, class Rad, int LPT>
constexpr const void *pass_c_ptr()
{
    if constexpr (LPT > 0)
        return (const void *)&k_pass_c<N, T, Rad, LPT>;
    else
        return nullptr;
}

template <int N, int T, class Rad>
constexpr const void *pass_ctma_ptr()
{
    constexpr int L = lpt_tma(N, T);
    if constexpr (L > 0)
        return (const void *)&k_pass_c_tma<N, T, Rad, L>;
    else
        return nullptr;
}

template <int N, int T, class Rad, int MODE>
constexpr const void *pass_j_tc_ptr()
{
    constexpr int mask = tc_mask_mode<Rad>(MODE);
    if constexpr (mask != 0 && N >= 128 && T * lpt_j(T) <= 512 && (T * lpt_j(T)) % 32 == 0)
        return (const void *)&k_pass_j_tc<N, T, Rad, lpt_j(T), mask>;
    else
        return nullptr;
}

template <int N, int T, class Rad, int MODE>
constexpr const void *pass_c_tc_ptr()
{
    constexpr int mask = tc_mask_mode<Rad>(MODE);
    if constexpr (mask != 0 && N >= 128 && T * 8 <= 512)
        return (const void *)&k_pass_c_tc<N, T, Rad, 8, mask>;
    else
        return nullptr;
}

} // namespace fft3

#define FFT3_KERNEL_ROW(ID, N, T, ...)                                                          \
    {ID,                                                                                        \
     (const void *)&fft3::k_pass_j<N, T, fft3::Radices<__VA_ARGS__>, fft3::lpt_j(T), false>,    \
     (const void *)&fft3::k_pass_j<N, T, fft3::Radices<__VA_ARGS__>, fft3::lpt_rot(T), true>,   \
     fft3::pass_c_ptr<N, T, fft3::Radices<__VA_ARGS__>, fft3::lpt_c(T, 16)>(),                  \
     fft3::pass_c_ptr<N, T, fft3::Radices<__VA_ARGS__>, fft3::lpt_c(T, 8)>(),                   \
     fft3::slab_l2_ptr<N, T, fft3::Radices<__VA_ARGS__>>(),                                    \
     {fft3::slab_blk_ptr<N, T, fft3::Radices<__VA_ARGS__>, 4>(),                               \
      fft3::slab_blk_ptr<N, T, fft3::Radices<__VA_ARGS__>, 8>()},                              \
     fft3::pass_ctma_ptr<N, T, fft3::Radices<__VA_ARGS__>>(),                                  \
     {fft3::pass_j_tc_ptr<N, T, fft3::Radices<__VA_ARGS__>, 0>(),                               \
      fft3::pass_j_tc_ptr<N, T, fft3::Radices<__VA_ARGS__>, 1>(),                               \
      fft3::pass_j_tc_ptr<N, T, fft3::Radices<__VA_ARGS__>, 2>()},                              \
     {fft3::pass_c_tc_ptr<N, T, fft3::Radices<__VA_ARGS__>, 0>(),                               \
      fft3::pass_c_tc_ptr<N, T, fft3::Radices<__VA_ARGS__>, 1>(),                               \
      fft3::pass_c_tc_ptr<N, T, fft3::Radices<__VA_ARGS__>, 2>()}},
