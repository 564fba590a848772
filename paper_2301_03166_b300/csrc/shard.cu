// shard.cu -- host-side split of a batch of independent ABFT factorizations
// over several GPUs (one process per GPU).  The matrices are independent, so
// the split needs no exchange on the data path: each GPU factors its share
// in one persistent launch and only the per-matrix statuses are gathered.
#include <algorithm>
#include <numeric>
#include <queue>
#include <vector>

#include "abft.h"

extern "C" {

int abft_batched_partition(int32_t count, const int64_t* n, int32_t G, int32_t* owner,
                           double* load) {
    if (count < 0) return -1;
    if (count > 0 && n == nullptr) return -2;
    for (int32_t i = 0; i < count; ++i)
        if (n[i] < 0) return -2;
    if (G < 1) return -3;
    if (count > 0 && owner == nullptr) return -4;
    // work of a matrix: its Cholesky flop count n^3 / 3
    std::vector<double> work(count);
    for (int32_t i = 0; i < count; ++i) work[i] = (double)n[i] * (double)n[i] * (double)n[i] / 3.0;
    std::vector<int32_t> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return work[a] > work[b]; });
    // longest processing time first: each matrix, largest first, to the GPU
    // with the least work so far (ties: the lower GPU index)
    using Slot = std::pair<double, int32_t>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int32_t g = 0; g < G; ++g) heap.push({0.0, g});
    std::vector<double> acc(G, 0.0);
    for (int32_t i : order) {
        Slot s = heap.top();
        heap.pop();
        owner[i] = s.second;
        acc[s.second] += work[i];
        heap.push({acc[s.second], s.second});
    }
    if (load)
        for (int32_t g = 0; g < G; ++g) load[g] = acc[g];
    return ABFT_OK;
}

}  // extern "C"
