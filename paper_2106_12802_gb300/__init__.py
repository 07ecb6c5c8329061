"""GB300-native multi-resolution sampling renderer (Hou et al., arXiv 2106.12802).

The compute path is libmrs.so (hand-written CUDA for sm_103a) behind the C ABI
in include/mrs.h; this package is a thin binding over it.  PyTorch is used for
device memory and streams only.
"""
from ._lib import MrsError, kernel_launches, library_path, load  # noqa: F401
from .render import (PROFILE_KERNELS, RenderContext, Scene, philox_uniforms, profile_enable,  # noqa: F401
                     profile_read, render, render_batch, render_stats)
from .fusion import (NPARAMS, NPARAMS_EXTRA, Net, conv3x3, conv3x3_dgrad, conv_set_ring, conv3x3_wgrad, gate, gate_async, get_grads, get_state, image_metrics,  # noqa: F401
                     load_checkpoint, save_checkpoint, set_state, train_step)
from .rdn import RDN  # noqa: F401
from .rdn import nparams as rdn_nparams  # noqa: F401
