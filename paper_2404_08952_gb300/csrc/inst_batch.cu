// Instantiations of the persistent batched stage (first- and second-order DOLINC stencils).
#include "launch.cuh"

namespace dol {

template <int DIM, int NV, int NS> static void reg(BatchFns *t)
{
    t[batch_index(DIM, NV, NS, PREC_F64)] = BatchPath<DIM, NV, NS, PREC_F64>::fns();
    t[batch_index(DIM, NV, NS, PREC_F32)] = BatchPath<DIM, NV, NS, PREC_F32>::fns();
    t[batch_index(DIM, NV, NS, PREC_BF16)] = BatchPath<DIM, NV, NS, PREC_BF16>::fns();
}

void register_batch(BatchFns *t)
{
    reg<2, 1, 1>(t);
    reg<2, 1, 2>(t);
    reg<2, 4, 1>(t);
    reg<2, 4, 2>(t);
    reg<3, 1, 1>(t);
    reg<3, 1, 2>(t);
    reg<3, 5, 1>(t);
    reg<3, 5, 2>(t);
}

}  // namespace dol
