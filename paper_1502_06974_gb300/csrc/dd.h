// Direction-dependent part of the library (scalar and 2x2 gains).
#pragma once

namespace gc {
void dd_release();
void ddpol_release();
}
