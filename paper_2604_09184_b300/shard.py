"""Row sharding of the single-system step across ranks (nb_set_shard).

Each rank, one process per GPU, holds the whole system and calls step() with
the same arguments. The library evaluates the O(N^2) kick (and the row-wise
force update after the direct solver) for the rank's block of target rows and
joins the blocks with two all-gathers per step: the trial kick's flagged
pairs, then the rows of the force. The all-gather is the callback made here,
over torch.distributed (NCCL for the CUDA buffers of a GPU run). Marshalling
only: packing and unpacking the blocks run in the library's kernels; this
module hands the library's raw exchange buffers to the collective.

The block layout, the partition of rows (nb_shard_rows) and the rank order
of the gathered blocks are fixed by the library; see include/nb.h.
"""
from __future__ import annotations

import ctypes as C

from . import nb as _nb

ALLGATHER_FN = _nb.ALLGATHER_FN  # the library's nb_allgather_fn


class _RawCuda:
    """Raw device memory as a CUDA array (no copy, no stream of its own)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1",
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None, "stream": None}


def device_bytes(ptr: int, nbytes: int):
    """A uint8 CUDA tensor over nbytes of device memory at ptr (no copy)."""
    import torch
    return torch.as_tensor(_RawCuda(ptr, nbytes), device="cuda")


def rows(n: int, rank: int, world: int) -> tuple[int, int]:
    """Target rows [row0, row1) of `rank` out of `world` for n bodies (the
    library's partition, nb_shard_rows)."""
    r0, r1 = C.c_int(), C.c_int()
    code = _nb.lib().nb_shard_rows(int(n), int(rank), int(world), C.byref(r0), C.byref(r1))
    if code != _nb.NB_OK:
        raise _nb.NbError(code, "nb_shard_rows")
    return r0.value, r1.value


def allgather_into(recv, send, group=None):
    """The exchange of a sharded step: recv (world x len(send) bytes) receives
    every rank's send block, rank r's at offset r x len(send)."""
    import torch.distributed as dist
    dist.all_gather_into_tensor(recv, send, group=group)


def torch_allgather(world: int, group=None):
    """An nb_allgather_fn over torch.distributed on this rank's device
    buffers. The collective is ordered on the stream the library passes (its
    own stream), so it follows the packing kernel and precedes the unpacking
    one. A failure is reported to the library, which fails the step."""
    import torch

    def fn(user, send, recv, nbytes, stream):
        try:
            st = (torch.cuda.ExternalStream(stream) if stream
                  else torch.cuda.default_stream())
            with torch.cuda.stream(st):
                allgather_into(device_bytes(recv, nbytes * world), device_bytes(send, nbytes),
                               group)
            return 0
        except Exception:  # noqa: BLE001 (reported to the library as a failed step)
            return -1

    return ALLGATHER_FN(fn)


class Shard:
    """Keeps a sharded system's exchange buffer and callback alive.

    system: an NBodySystem; rank, world: this process's place; fn: an
    ALLGATHER_FN (torch_allgather by default, needs an initialised
    torch.distributed process group)."""

    def __init__(self, system, rank: int, world: int, fn=None, group=None):
        import torch
        L = _nb.lib()
        self.system = system
        self.rank, self.world = int(rank), int(world)
        self.fn = fn if fn is not None else (torch_allgather(world, group) if world > 1 else None)
        nbytes = int(L.nb_shard_buffer_bytes(system._h, self.world))
        if nbytes == 0:
            raise _nb.NbError(_nb.NB_E_INVALID, "nb_shard_buffer_bytes")
        self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.buf.data_ptr()
        code = L.nb_set_shard(system._h, self.rank, self.world,
                              self.fn if self.fn is not None else ALLGATHER_FN(), None,
                              C.c_void_p(base + (-base) % 256), nbytes)
        if code != _nb.NB_OK:
            raise _nb.NbError(code, _nb.lib().nb_last_error(system._h).decode())
        self.row0, self.row1 = rows(system.n, self.rank, self.world)

    def release(self):
        """Back to the unsharded step (the buffer may then be freed)."""
        _nb.lib().nb_set_shard(self.system._h, 0, 1, ALLGATHER_FN(), None, None, 0)
