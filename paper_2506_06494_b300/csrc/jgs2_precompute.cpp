// Offline stage of JGS2 (Secs. 5-6) on the host: placeholder until the sparse factorisation
// lands; jgs2_precompute reports that it is unavailable.
#include "../../include/jgs2.h"
#include "jgs2_host.h"

extern "C" jgs2_status jgs2_precompute(jgs2_mesh* mesh, const jgs2_precompute_opts* opts) {
  (void)mesh;
  (void)opts;
  return jgs2::fail(JGS2_EINVAL, "jgs2_precompute: not built yet");
}
