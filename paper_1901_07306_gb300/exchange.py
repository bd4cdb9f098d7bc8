"""Exchange between watch points on different GPUs or boxes (Sec. 4.2).

Every watch point (WP) ships its SEAV and LDCA to the global server (GS),
which ORs them into the global sketch.  Across processes this module only
moves bytes with ``torch.distributed`` tensor collectives; all sketch
arithmetic (the OR, the detect) runs in the library on the GPU.

Two forms:
  * device form (NCCL): each rank copies its router's sketch into a device
    tensor (``sp_copy_sketch``), the tensors are all-gathered in device
    memory, and a rank ORs the peers' images into a router
    (``sp_merge_device``).  Nothing passes through the host.
  * host form (any backend, e.g. gloo between boxes): checksummed
    ``sp_export`` images are all-gathered as uint8 tensors, imported into
    spare router slots (``sp_import``, checksum-verified) and OR-merged on the
    GPU (``sp_merge``).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def _device_for(group=None) -> torch.device:
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def all_gather_images(image: bytes, group=None) -> list[bytes]:
    """Every rank's sp_export image, in rank order.  Images of one parameter
    set have the same size on every rank (checked), so they travel as one
    uint8 tensor per rank through all_gather_into_tensor."""
    world = dist.get_world_size(group)
    dev = _device_for(group)
    local = torch.from_numpy(np.frombuffer(image, np.uint8).copy()).to(dev)
    sizes = torch.zeros(world, dtype=torch.int64, device=dev)
    dist.all_gather_into_tensor(sizes, torch.tensor([local.numel()], dtype=torch.int64, device=dev), group=group)
    if not bool((sizes == local.numel()).all()):
        raise ValueError(f"sketch images differ in size across ranks: {sizes.tolist()}")
    out = torch.empty(world * local.numel(), dtype=torch.uint8, device=dev)
    dist.all_gather_into_tensor(out, local, group=group)
    host = out.cpu().numpy().reshape(world, -1)
    return [host[r].tobytes() for r in range(world)]


def merge_remote_images(sp_module, ctx: int, images: list[bytes], first_slot: int, dst_router: int) -> int:
    """Host form: imports the images into routers first_slot, first_slot + 1,
    ... and OR-merges them into dst_router on the GPU.  Returns the first
    failing sp_import status, or 0."""
    slots = []
    for i, img in enumerate(images):
        rc = sp_module.sp_import(ctx, first_slot + i, img)
        if rc != 0:
            return rc
        slots.append(first_slot + i)
    sp_module.sp_merge(ctx, slots, dst_router)
    return 0


def all_gather_sketches(sp_module, ctx: int, router: int, group=None) -> torch.Tensor:
    """Device form: a [world, n] uint8 CUDA tensor holding every rank's device
    image of `router` (sp_copy_sketch), gathered over NCCL.  The copy is
    issued on the context's stream, which must be the current torch stream
    (NCCL orders its collective after the current stream's work)."""
    world = dist.get_world_size(group)
    n = sp_module.sp_copy_sketch_bytes(ctx)
    local = torch.empty(n, dtype=torch.uint8, device="cuda")
    sp_module.sp_copy_sketch(ctx, router, local)
    out = torch.empty(world * n, dtype=torch.uint8, device="cuda")
    dist.all_gather_into_tensor(out, local, group=group)
    return out.view(world, n)


def merge_gathered(sp_module, ctx: int, gathered: torch.Tensor, dst_router: int, skip=()) -> None:
    """ORs the gathered device images (rows of `gathered`, except the ranks
    in `skip`, e.g. the local one already in dst_router) into dst_router."""
    rows = [gathered[r] for r in range(gathered.shape[0]) if r not in set(skip)]
    sp_module.sp_merge_device(ctx, rows, dst_router)


def reduce_max(value: float, group=None) -> float:
    """Max over ranks (the benchmark's whole-job time), on the backend's device."""
    if not dist.is_available() or not dist.is_initialized():
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device_for(group))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
