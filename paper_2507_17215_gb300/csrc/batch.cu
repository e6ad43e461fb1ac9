// Batched queries. This first form answers the queries one after another on the
// stream; it defines the results the shared-probe batch kernel must reproduce.
#include "internal.cuh"

namespace folty {

void run_query_batch(folty_graph* g, const folty_query_params* qs, int nq, folty_result* outs,
                     cudaStream_t s) {
    for (int i = 0; i < nq; i++) run_query(g, qs[i], &outs[i], s);
}

}  // namespace folty
