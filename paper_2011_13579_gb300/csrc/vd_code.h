// Internal definition of the opaque vd_code object (shared by the C-ABI sources).
#pragma once
#include <cstdint>
#include "vd_launch.h"

struct vd_code {
    int K, beta;
    uint32_t gens[4];
    int period;
    uint8_t punct[4][8];
    int kept_per_period;
    int kept_prefix[9];      // kept values before phase p within a period
    bool punctured;
    vd::CodeKind kind;
};

// Sets the calling thread's message returned by vd_last_error().
void vd_internal_set_error(const char *msg);
