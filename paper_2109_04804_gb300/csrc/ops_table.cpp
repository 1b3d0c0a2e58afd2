// Dispatch from (law, dim, P, node family) to the compiled operator launchers.
#include "hbpc_internal.h"
#include "ops_units.h"

namespace hbpc {

#define HBPC_DECL(name, law, dim, lm, gm) bool get_ops_unit_##name(int P, bool lgl, OpsTable& t);
HBPC_OPS_UNITS(HBPC_DECL)
#undef HBPC_DECL

bool get_ops(int law, int dim, int P, bool lobatto, OpsTable& out) {
  out = OpsTable{};
#define HBPC_TRY(name, l, d, lm, gm)                                              \
  if (law == l && dim == d && (((lobatto ? (lm) : (gm)) >> P) & 1))              \
    return get_ops_unit_##name(P, lobatto, out);
  HBPC_OPS_UNITS(HBPC_TRY)
#undef HBPC_TRY
  return false;
}

}  // namespace hbpc
