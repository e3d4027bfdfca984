// Direction-dependent (CohJones) part of the library.
#pragma once

namespace gc {
void dd_release();
}
