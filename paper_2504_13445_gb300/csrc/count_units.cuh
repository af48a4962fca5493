// Decoding of the counting pass's work units (the list k_build_units writes; device side).
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace rkm {

// Local unit lw of a counting stage -> item tile T and user tiles [ut0, ut1).  Units are
// tile-major: unit_off[j] is the first unit of tile t_begin + j, whose units are its groups of
// `group` user tiles in order.  Every unit holds at least one user tile.
__device__ __forceinline__ void decode_count_unit(const CountArgs& a, unsigned lw, int& T, int64_t& ut0,
                                                  int64_t& ut1) {
    int lo = 0, hi = a.st->t_end - a.t_begin;  // unit_off has hi + 1 entries
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.unit_off[mid] <= lw) lo = mid; else hi = mid;
    }
    T = a.t_begin + lo;
    const int g = (int)(lw - a.unit_off[lo]);
    const int64_t nT = a.nprefix[T];
    const int64_t all = (nT + BU - 1) / BU;
    ut0 = (int64_t)g * a.group;
    ut1 = ut0 + a.group;
    if (ut1 > all) ut1 = all;
}

}  // namespace rkm
