"""FP64 CPU oracle for the 2D SGN hot path. Test infrastructure only: the GPU
library never imports it."""
from . import sgn_oracle  # noqa: F401
