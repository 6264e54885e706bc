"""GB300-native hot path of NARVis (arXiv 2407.19097): a multi-attribute point rasterizer and a
neural deferred renderer as hand-written sm_103a CUDA behind the C ABI in include/nrv.h.
`autograd` (imported on demand, it needs torch) puts the network behind torch.autograd."""
from . import nrv  # noqa: F401
from .build_lib import build  # noqa: F401
