// rtlbfs_worklist.h -- host-side ordering of a step's work list (plain C++,
// no CUDA types, so that it also builds into host-only unit tests).
#pragma once

#include <cstddef>
#include <vector>

namespace rtlbfs {

// Reorder units [b, end) of a work list so that those for which edge(u) is
// true are spaced evenly among the others; each group keeps its own order.
// Unit k of the range is an edge unit exactly when floor((k+1) ne / n)
// exceeds floor(k ne / n) (ne edge units of n), so between two edge units
// there are floor or ceil of (n - ne) / ne others, and blocks handed out to
// the SMs in list order get the edge units as evenly as the count allows.
template <class T, class Edge>
void spread_units(std::vector<T>& t, std::size_t b, Edge edge)
{
    if (b >= t.size()) return;
    std::vector<T> e, in;
    for (std::size_t k = b; k < t.size(); ++k) (edge(t[k]) ? e : in).push_back(t[k]);
    const long long ne = (long long)e.size(), n = ne + (long long)in.size();
    std::size_t ie = 0, ii = 0;
    for (long long k = 0; k < n; ++k) {
        const bool take_edge = (k + 1) * ne / n > k * ne / n;
        t[b + (std::size_t)k] = take_edge ? e[ie++] : in[ii++];
    }
}

}  // namespace rtlbfs
