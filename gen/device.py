"""Seeded synthetic workloads generated on the GPU (bit-identical to gen/host.py).

Returns CUDA tensors with int32 / int64 dtype holding the uint32 / uint64 bits.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from gen import host as H

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "libahsgen.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise ImportError(f"{_LIB} missing: run gen/build.py")
        L = ctypes.CDLL(_LIB)
        u64, vp = ctypes.c_uint64, ctypes.c_void_p
        L.gen_uniform_u32.argtypes = [vp, u64, u64, u64, u64, u64, vp]
        L.gen_zipf_u32.argtypes = [vp, u64, u64, u64, vp, vp, ctypes.c_uint, u64, vp]
        L.gen_ramp_steps.argtypes = [vp, u64, u64, u64, vp]
        L.gen_ramp_replace.argtypes = [vp, u64, u64, u64, u64, u64, vp]
        L.gen_swaps_u32.argtypes = [vp, u64, u64, u64, u64, vp]
        L.gen_batch_u32.argtypes = [vp, vp, vp, ctypes.c_uint, u64, vp, ctypes.c_uint, vp]
        L.gen_gaussian_i32.argtypes = [vp, u64, u64, u64, ctypes.c_longlong, u64, vp]
        L.gen_replace_u32.argtypes = [vp, u64, u64, u64, u64, vp]
        L.gen_kmer_u64.argtypes = [vp, u64, u64, u64, u64, vp]
        L.gen_batch_swaps.argtypes = [vp, vp, vp, ctypes.c_uint, u64, vp]
        _lib = L
    return _lib


def _st():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ok(rc):
    if rc != 0:
        raise RuntimeError(f"generator launch failed ({rc})")


def uniform_u32(n, seed, stream, m, start=0):
    import torch
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    _ok(lib().gen_uniform_u32(out.data_ptr(), n, seed, stream, m, start, _st()))
    return out


def zipf_u32(n, seed, stream_values, stream_ranks, n_values=1024, s=1.1, start=0):
    import torch
    cdf = torch.from_numpy(H.zipf_cdf(n_values, s)).cuda()
    vals = torch.from_numpy(H.zipf_values(seed, stream_values, n_values).view(np.int32)).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    _ok(lib().gen_zipf_u32(out.data_ptr(), n, seed, stream_ranks, cdf.data_ptr(), vals.data_ptr(),
                           n_values, start, _st()))
    torch.cuda.synchronize()
    return out


def gaussian_i32(n, seed, stream, k, start=0):
    """int32 keys shaped like N(0, k/4) (as gen.host.gaussian_i32)."""
    import torch
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    _ok(lib().gen_gaussian_i32(out.data_ptr(), n, seed, stream, H.gauss_sigma_q16(k), start, _st()))
    return out


def kmer_u64(n, seed, stream, start=0):
    """uint64 60-bit k-mer keys (int64 tensor; as gen.host.kmer_u64)."""
    import torch
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    _ok(lib().gen_kmer_u64(out.data_ptr(), n, seed, stream, start, _st()))
    return out


def replace_u32(a, seed, stream, thresh53=H.REPLACE_1PCT_53):
    _ok(lib().gen_replace_u32(a.data_ptr(), a.numel(), seed, stream, thresh53, _st()))
    return a


def request_keys(seed, rid, kind, n):
    """Keys of a library-generated served request (as gen.host.request_keys)."""
    s0 = H.request_stream(rid, 0)
    if kind == 0:
        return uniform_u32(n, seed, s0, 4096)
    if kind == 1:
        return zipf_u32(n, seed, H.request_stream(rid, 1), s0)
    if kind == 2:
        return uniform_u32(n, seed, s0, 1 << 32)
    return replace_u32(sorted_u32(uniform_u32(n, seed, s0, 1 << 32)), seed, H.request_stream(rid, 2))


def sorted_u32(x):
    """Ascending order of uint32 bits held in an int32 tensor."""
    import torch
    s = torch.sort(x.to(torch.int64) & 0xFFFFFFFF).values
    return s.to(torch.int32)


def swaps_u32(a, n_swaps, seed, stream):
    _ok(lib().gen_swaps_u32(a.data_ptr(), a.numel(), n_swaps, seed, stream, _st()))
    return a


def config1(n=H.N_CFG1):
    return uniform_u32(n, H.SEED_CFG1, 0, 256)


def config2(variant, n=H.N_CFG2, seed=H.SEED_CFG2):
    import torch
    if variant == "a":
        return uniform_u32(n, seed, 1, 4096)
    if variant == "b":
        return zipf_u32(n, seed, 2, 3)
    if variant == "c":
        return uniform_u32(n, seed, 4, 1 << 32)
    base = sorted_u32(uniform_u32(n, seed, 4, 1 << 32))
    if variant == "d":
        return base
    if variant == "e":
        return swaps_u32(base, n // 100, seed, 5)
    if variant == "f":
        return torch.flip(base, dims=[0]).contiguous()
    raise ValueError(variant)


def config3(n=H.N_CFG3, seed=H.SEED_CFG3, t0=1_700_000_000_000_000_000, max_step=1000):
    """uint64 ramp keys (int64 tensor) and uint32 payload = index (int32 tensor)."""
    import torch
    steps = torch.empty(n, dtype=torch.int64, device="cuda")
    _ok(lib().gen_ramp_steps(steps.data_ptr(), n, seed, max_step + 1, _st()))
    t = torch.cumsum(steps, 0) + t0
    last = int(t[-1].item())
    rng = last - t0 + 1
    _ok(lib().gen_ramp_replace(t.data_ptr(), n, seed, H.REPLACE_53, t0, rng % (1 << 64), _st()))
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    return t, vals


def config4(n_seg=100_000, seed=H.SEED_CFG4, lo=16, hi=1 << 20, sort_chunk_keys=1 << 27):
    """Batch of uneven segments: (keys int32 tensor, offsets np.uint64, lengths, types).

    Types index gen.host.SEG_TYPES = (a, b, c, e); each segment is generated
    from (seed, segment id) exactly as gen.host.config4_segment.  Type (e)
    segments are sorted (PyTorch, by (segment, key)) and then swapped."""
    import torch
    lengths, types, offsets = H.config4_layout(n_seg, seed, lo, hi)
    total = int(offsets[-1])
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    d_offs = torch.from_numpy(offsets.view(np.int64)).cuda()
    d_types = torch.from_numpy(types.astype(np.uint8)).cuda()
    cdf = torch.from_numpy(H.zipf_cdf(1024, 1.1)).cuda()
    _ok(lib().gen_batch_u32(out.data_ptr(), d_offs.data_ptr(), d_types.data_ptr(), n_seg, seed,
                            cdf.data_ptr(), 1024, _st()))
    # sort every type-(e) segment: groups of consecutive e-segments by key size
    e_segs = np.nonzero(types == 3)[0]
    i = 0
    while i < len(e_segs):
        j, keys = i, 0
        while j < len(e_segs) and (j == i or keys + int(lengths[e_segs[j]]) <= sort_chunk_keys):
            keys += int(lengths[e_segs[j]])
            j += 1
        parts = [out[int(offsets[s]):int(offsets[s + 1])] for s in e_segs[i:j]]
        cat = torch.cat(parts).to(torch.int64) & 0xFFFFFFFF
        tag = torch.repeat_interleave(torch.arange(j - i, device="cuda", dtype=torch.int64),
                                      torch.tensor([int(lengths[s]) for s in e_segs[i:j]],
                                                   device="cuda"))
        srt = torch.sort((tag << 32) | cat).values & 0xFFFFFFFF
        at = 0
        for s in e_segs[i:j]:
            L = int(lengths[s])
            out[int(offsets[s]):int(offsets[s + 1])] = srt[at:at + L].to(torch.int32)
            at += L
        i = j
    d_e = torch.from_numpy(e_segs.astype(np.uint32).view(np.int32)).cuda()
    _ok(lib().gen_batch_swaps(out.data_ptr(), d_offs.data_ptr(), d_e.data_ptr(), len(e_segs), seed,
                              _st()))
    torch.cuda.synchronize()
    return out, offsets, lengths, types
