"""Host-side exchange between watch points on different GPUs or boxes.

Sec. 4.2 ships every watch point's SEAV and LDCA to a global server.  Across
processes this module only moves bytes: each rank exports its sketch image
(``sp_export``), the images are all-gathered over ``torch.distributed``
(gloo or NCCL), and the receiver imports them into spare router slots
(``sp_import``, checksum-verified) and ORs them on its GPU with ``sp_merge``.
No sketch arithmetic happens here.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def all_gather_images(image: bytes, group=None) -> list[bytes]:
    """Every rank's sketch image, in rank order."""
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, bytes(image), group=group)
    return out


def reduce_max(value: float, group=None) -> float:
    """Max over ranks (the benchmark's whole-job time), on the backend's device."""
    if not dist.is_available() or not dist.is_initialized():
        return value
    backend = dist.get_backend(group)
    device = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def merge_remote_images(sp_module, ctx: int, images: list[bytes], first_slot: int, dst_router: int) -> int:
    """Imports the images into routers first_slot, first_slot + 1, ... and
    OR-merges them into dst_router on the GPU.  Returns the first failing
    sp_import status, or 0."""
    slots = []
    for i, img in enumerate(images):
        rc = sp_module.sp_import(ctx, first_slot + i, img)
        if rc != 0:
            return rc
        slots.append(first_slot + i)
    sp_module.sp_merge(ctx, slots, dst_router)
    return 0
