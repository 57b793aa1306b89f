// Equal-work partition of a family's pair range over several GPUs (host only).
//
// The pairs of the posterior stage are independent (paper, Methods, stage I:
// posteriors and distances are computed for all pairs of sequences), so one
// family is split into contiguous ranges of the linear pair order, one per
// rank, each holding about the same work.  The work of pair (a, b) is its cell
// count m n, the unit of the stage's cost.
#include "../../include/qp.h"
#include "qp_host.h"

#include <vector>

extern "C" int qp_split_pairs(int32_t k, const int64_t* offsets, int32_t n_parts, int64_t* bounds) {
    using namespace qph;
    if (!offsets || !bounds) return fail(QP_EINVAL, "offsets or bounds is NULL");
    if (k < 2 || k > kMaxK) return fail(QP_EINVAL, "k = %d outside [2, %d]", k, kMaxK);
    const int64_t P = (int64_t)k * (k - 1) / 2;
    if (n_parts < 1 || (int64_t)n_parts > P)
        return fail(QP_EINVAL, "n_parts = %d outside [1, %lld] (every part needs a pair)", n_parts, (long long)P);
    if (offsets[0] != 0) return fail(QP_EINVAL, "offsets[0] must be 0");
    std::vector<int64_t> len(k);
    for (int a = 0; a < k; ++a) {
        len[a] = offsets[a + 1] - offsets[a];
        if (len[a] < 1) return fail(QP_EINVAL, "sequence %d is empty", a);
    }
    // cumulative work in the linear order p = a k - a(a+1)/2 + (b - a - 1):
    // the pairs of row a are (a, a+1), ..., (a, k-1)
    std::vector<double> cum(P + 1);
    cum[0] = 0.0;
    int64_t p = 0;
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b, ++p) cum[p + 1] = cum[p] + (double)len[a] * (double)len[b];
    const double total = cum[P];
    bounds[0] = 0;
    bounds[n_parts] = P;
    int64_t lo = 0;
    for (int i = 1; i < n_parts; ++i) {
        // the boundary whose prefix work is nearest to i / n_parts of the
        // total, keeping every part non-empty
        const double target = total * (double)i / (double)n_parts;
        int64_t b = lo + 1;
        const int64_t hi = P - (n_parts - i);          // leave a pair for every later part
        while (b < hi && cum[b + 1] <= target) ++b;
        if (b < hi && target - cum[b] > cum[b + 1] - target) ++b;
        bounds[i] = b;
        lo = b;
    }
    return QP_OK;
}
