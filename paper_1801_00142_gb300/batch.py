"""Many independent XTRG runs on one GPU through ``xtrg_batch_run``.

The native runner cuts one workspace into equal slots and drives each slot
with a host thread and a stream of its own (see include/xtrg.h); this module
only sizes and allocates that workspace with PyTorch and marshals the
arguments.
"""
from __future__ import annotations

import torch

from . import _lib


def run_batch(items, max_concurrent=0, device="cuda:0", memory_fraction=0.8):
    """items: list of (H_dims, H_sites, n_doublings, config keywords of
    ``_lib.make_config``).  Returns one list of observables rows per item."""
    if not torch.cuda.is_available():
        raise RuntimeError("the batch runner needs a CUDA device")
    Hs = [_lib.MpoArgs(d, s) for d, s, _, _ in items]
    cfgs = [_lib.make_config(**kw) for _, _, _, kw in items]
    nds = [nd for _, _, nd, _ in items]
    dev = torch.device(device)
    slots, slot_bytes = _lib.xtrg_batch_plan(Hs, cfgs, 1 << 62, max_concurrent)
    free, _ = torch.cuda.mem_get_info(dev)
    slots = max(1, min(slots, int(free * memory_fraction) // slot_bytes))
    nbytes = slots * slot_bytes
    with torch.cuda.device(dev):
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        stream = torch.cuda.current_stream(dev)
    ptr = (ws.data_ptr() + 255) // 256 * 256
    rows = _lib.xtrg_batch_run(Hs, cfgs, nds, ptr, nbytes, slots, stream.cuda_stream)
    torch.cuda.synchronize(dev)
    del ws
    return rows
