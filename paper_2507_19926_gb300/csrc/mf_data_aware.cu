// Data-aware variant (paper Sec. 5) -- placeholder until the kernel lands.
#include <cstdio>

#include "mf_registry.h"

namespace mf {
int d1_supported(int, int, bool) { return 0; }
int d1_supported_tile(int, int, bool, int) { return 0; }
int d1_default_tile(int, int, bool) { return 0; }
int d1_launch(const ImgArgs &, int, int, int, int, cudaStream_t) {
    set_error("data-aware variant not built");
    return MF_ERR_UNSUPPORTED;
}
int d1_describe(int k, int, bool, int tile, char *buf, size_t n) {
    snprintf(buf, n, "data-aware k=%d tile=%d", k, tile);
    return MF_OK;
}
}  // namespace mf
