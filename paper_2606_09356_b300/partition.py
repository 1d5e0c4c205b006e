"""Chain partition of one system: the system's chains split into contiguous
ranges, one handle per range (one GPU each), and one exchange per step: the
partial density counts summed over all partitions (the decomposition whose
density-field communication limits SOMA's own multi-GPU scaling, Sec. 2.2).

The library does the moves and the partial histogram; the sum is the
caller's: a torch.distributed all-reduce across processes (NCCL between GPUs,
gloo on CPU), or, for partitions on one GPU, a plain sum of their buffers.
"""


def chain_range(n_poly, rank, world):
    """The logical chains [begin, end) of partition `rank` of `world`:
    contiguous ranges whose sizes differ by at most one chain."""
    if not (0 <= rank < world) or n_poly < world:
        raise ValueError("need 0 <= rank < world <= n_poly")
    q, r = divmod(int(n_poly), int(world))
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


class _DeviceWords:
    """A device buffer of uint32 words seen as int32 through the CUDA array
    interface (sums of counts below 2^31 are the same in either type)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<i4", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def counts_tensor(handle):
    """The counts the handle's next step reads, as an int32 CUDA tensor on
    the handle's GPU that aliases the library's buffer (valid until the
    handle steps or re-bins)."""
    import torch
    ptr, n = handle.exchange_counts()
    with torch.cuda.device(handle.device):
        return torch.as_tensor(_DeviceWords(ptr, n), device=f"cuda:{handle.device}")


def all_reduce_sum(group=None):
    """The exchange across processes: torch.distributed's all-reduce (sum)
    of the counts tensor, ordered on the current CUDA stream."""
    import torch.distributed as dist

    def reduce(t):
        dist.all_reduce(t, group=group)
    return reduce


def _stream(stream):
    """The torch CUDA stream the step and the exchange share: not the legacy
    default stream, whose raw handle (0) the library would read as "the
    handle's own stream", unordered with torch's work."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    if st.cuda_stream == 0:
        raise ValueError("partition steps need a non-default CUDA stream (torch.cuda.Stream())")
    return st


def exchange(handle, reduce, stream=None):
    """Replace the handle's partial counts by their sum over all partitions,
    on `stream` (a torch.cuda.Stream; default: the current one); call after
    creating the handle, after every step and after anything that re-bins
    (set_state, place, set_chain_types)."""
    import torch
    with torch.cuda.stream(_stream(stream)):
        reduce(counts_tensor(handle))


def step(handle, reduce, stream=None):
    """One Monte Carlo step of a partition followed by the exchange, both on
    `stream` (a non-default torch.cuda.Stream; default: the current one)."""
    st = _stream(stream)
    handle.mc_steps(1, stream=st.cuda_stream)
    exchange(handle, reduce, st)


def sum_on_one_device(handles, stream=None):
    """The exchange of several partitions held on one GPU: every partition's
    buffer becomes the sum of all of them, on `stream` (as for step)."""
    import torch
    with torch.cuda.stream(_stream(stream)):
        ts = [counts_tensor(h) for h in handles]
        total = ts[0].clone()
        for t in ts[1:]:
            total += t
        for t in ts:
            t.copy_(total)
