// Instantiations of the stage paths for dim = 2, 4 variable(s).
#include "launch.cuh"

namespace dol {

template <int NS> static void reg(PathFns *t)
{
    t[path_index(2, 4, NS, PREC_F64)] = Path<2, 4, NS, PREC_F64>::fns();
    t[path_index(2, 4, NS, PREC_F32)] = Path<2, 4, NS, PREC_F32>::fns();
    t[path_index(2, 4, NS, PREC_BF16)] = Path<2, 4, NS, PREC_BF16>::fns();
}

void register_paths_d2e(PathFns *t)
{
    reg<1>(t);
    reg<2>(t);
    reg<3>(t);
    reg<4>(t);
}

}  // namespace dol
