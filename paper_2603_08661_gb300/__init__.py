"""GB300-native edge-guided densification path of ImprovedGS+ (arXiv 2603.08661).

The compute lives in libgsp.so (C ABI, include/gsp.h), built for sm_103a by
`paper_2603_08661_gb300.build`.  This package is its thin Python binding:

* edge_map            - Sec. 2.1 edge-importance maps (fused or plain)
* Renderer            - tile-binned splatting forward / adjoint with edge score
* topk_mask, las_split - Sec. 2.2 selection and Long-Axis-Split (Alg. 1-2)
* GaussianRenderL1    - torch.autograd.Function over the forward / adjoint
* autotune.tune       - picks the fastest compositing variants for a workload
* DensifyLoop         - device-resident loop: fwd/L1/bwd+score/SGD, top-k + LAS events
* ShardedRenderer     - view-sharded forward/adjoint over the ranks of a process
                        group, one all-reduce of gradients, scores and loss

Importing fails loudly when libgsp.so is missing; there is no CPU fallback.
"""
from . import _lib

_lib.load()

from .api import (LAS_CONFIG, LAS_PAPER, GaussianSet, Renderer, StageTimer, camera_struct,  # noqa: E402,F401
                  edge_map, image_desc, las_split, launch_count, new_status, pitched_image,
                  raise_on_device_status, sample_mask, select_mask, topk_mask, topk_mask_gated)
from .autograd import GaussianRenderL1  # noqa: E402,F401
from . import autotune  # noqa: E402,F401
from .loop import DensifyLoop  # noqa: E402,F401
from .sharded import FlatGrads, ShardedRenderer, all_reduce_flat, partition_views  # noqa: E402,F401
