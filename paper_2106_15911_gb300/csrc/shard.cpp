// shard.cpp -- temporal decomposition of the space-time FMM over several GPUs (Section 4):
// the owner of every cluster of the binary temporal tree (the "scheduling tree") and the
// one-directional messages of a distributed matrix-vector product.
//
// Owners (Section 4.1, the three rules), with P ranks and L0 = ceil(log2 P):
//   * levels >= L0 hold at least P clusters: they are given to the ranks in ascending order and as
//     evenly as possible (rank of cluster k at level l = floor(k P / 2^l));
//   * level L0 - 1: a cluster goes to the rank of its left child (the left child's interaction
//     list is the smaller one, Eq. 03:ILtemp);
//   * levels l < L0 - 1: the ranks are split into 2^l groups of consecutive ranks; cluster k takes,
//     from group k, the rank that owns the fewest clusters so far (lowest rank on ties).
// Messages (Section 4.2: the M-, M2L-, L- and N-lists and their dependencies): the moments of a
// cluster go to the owner of its parent (M2M) and to the owners of the clusters whose interaction
// list holds it (M2L: target k + 2, and k + 3 when k is even); the locals of a cluster go to the
// owners of its two children (L2L); the input of a leaf interval goes to the owner of the next
// leaf interval (nearfield: N(I_k) = {I_{k-1}, I_k}).  Each (kind, cluster, destination) is sent
// once.  Everything here is host logic; one process per GPU would post these messages as NCCL
// send / recv of the per-interval slabs (no collective: the result stays distributed).
#include <cstdint>
#include <set>
#include <tuple>
#include <vector>

#include "handle.h"

namespace {

int ceil_log2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// owner[(1 << l) - 1 + k] of cluster k on level l, l = 0 .. levels
std::vector<int> shard_owners(int levels, int P)
{
    std::vector<int> owner((size_t(1) << (levels + 1)) - 1, 0);
    std::vector<long long> count(P, 0);
    const int L0 = ceil_log2(P);
    auto at = [&](int l, int k) -> int & { return owner[(size_t(1) << l) - 1 + k]; };
    for (int l = levels; l >= 0; --l) {
        const int n = 1 << l;
        for (int k = 0; k < n; ++k) {
            int r;
            if (l >= L0) {
                r = (int)((long long)k * P / n);
            } else if (l == L0 - 1 && l < levels) {
                r = at(l + 1, 2 * k);
            } else {
                // group k of the ranks split into n consecutive groups
                const int g0 = (int)((long long)k * P / n), g1 = (int)((long long)(k + 1) * P / n);
                r = g0;
                for (int q = g0; q < g1; ++q)
                    if (count[q] < count[r]) r = q;
            }
            at(l, k) = r;
            count[r]++;
        }
    }
    return owner;
}

}  // namespace

extern "C" {

int pfmm_shard_owners(int32_t levels, int32_t nranks, int32_t *owner)
{
    if (levels < 0 || levels > 24 || nranks < 1 || !owner)
        return pfmm::set_error(PFMM_ERR_INVALID_ARG, "invalid pfmm_shard_owners arguments");
    std::vector<int> o = shard_owners(levels, nranks);
    for (size_t i = 0; i < o.size(); ++i) owner[i] = o[i];
    return PFMM_OK;
}

int pfmm_shard_messages(int32_t levels, int32_t nranks, int32_t *msgs, int64_t cap, int64_t *count)
{
    if (levels < 0 || levels > 24 || nranks < 1 || !count || cap < 0 || (cap > 0 && !msgs))
        return pfmm::set_error(PFMM_ERR_INVALID_ARG, "invalid pfmm_shard_messages arguments");
    std::vector<int> o = shard_owners(levels, nranks);
    auto own = [&](int l, int k) { return o[(size_t(1) << l) - 1 + k]; };
    std::set<std::tuple<int, int, int, int>> seen;  // (kind, level, interval, dst)
    std::vector<int32_t> out;
    auto add = [&](int kind, int l, int k, int dst) {
        const int src = own(l, k);
        if (src == dst || !seen.insert(std::make_tuple(kind, l, k, dst)).second) return;
        out.insert(out.end(), {kind, l, k, src, dst});
    };
    for (int l = levels; l >= 0; --l) {
        const int n = 1 << l;
        for (int k = 0; k < n; ++k) {
            // moments: to the parent's owner (M2M) and to the M2L targets (levels >= 2)
            if (l >= 3) add(PFMM_MSG_MOMENTS, l, k, own(l - 1, k >> 1));
            if (l >= 2) {
                if (k + 2 < n) add(PFMM_MSG_MOMENTS, l, k, own(l, k + 2));
                if (k % 2 == 0 && k + 3 < n) add(PFMM_MSG_MOMENTS, l, k, own(l, k + 3));
            }
            // locals: to the children's owners (L2L)
            if (l < levels && l >= 2) {
                add(PFMM_MSG_LOCALS, l, k, own(l + 1, 2 * k));
                add(PFMM_MSG_LOCALS, l, k, own(l + 1, 2 * k + 1));
            }
            // input halo of the nearfield: leaf k to the owner of leaf k + 1
            if (l == levels && k + 1 < n) add(PFMM_MSG_INPUT, l, k, own(l, k + 1));
        }
    }
    *count = (int64_t)out.size() / 5;
    for (int64_t i = 0; i < (int64_t)out.size() && i < 5 * cap; ++i) msgs[i] = out[(size_t)i];
    return PFMM_OK;
}

}  // extern "C"
