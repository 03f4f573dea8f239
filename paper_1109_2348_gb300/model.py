"""Learned CDF model for the learned bucketing: training and compilation.

Every step runs in the CUDA library: the plain sorter produces the training
samples (bwt_model_samples), the library's own FP32 forward/backward/Adam
kernels train the MLP (bwt_model_train), and bisection with the forward
kernel compiles it into the sorted splitter table (bwt_model_compile). This
module only draws the seeded random inputs (sample positions, minibatch
orders, initial weights -- all from ``datagen``) and passes pointers.

Training recipe: 10^6 samples drawn uniformly over all rotations of 100
order-3 Markov blocks (seeds 5000..5099), Adam with lr 1e-3 and batch 4096,
initial weights uniform in +-1/sqrt(fan_in), biases 0. The 8 input bytes are
normalised through the CDF of byte values in the training blocks
(bwt_model_byte_norm), so byte values the data never holds add nothing to
the model's CDF and the compiled splitters land where keys exist.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import Plan, _lib, datagen
from ._lib import check

NPARAMS = _lib.MLP_NPARAMS
SPLITTERS = _lib.SPLITTERS


def init_params(seed: int) -> np.ndarray:
    """Uniform +-1/sqrt(fan_in) weights, zero biases (float32, library layout)."""
    u = datagen.uniform_unit(seed, NPARAMS) * 2.0 - 1.0
    p = np.zeros(NPARAMS, dtype=np.float64)
    p[0:256] = u[0:256] / np.sqrt(8.0)            # W1[32][8]
    p[288:1312] = u[288:1312] / np.sqrt(32.0)     # W2[32][32]
    p[1344:1376] = u[1344:1376] / np.sqrt(32.0)   # W3[32]
    return p.astype(np.float32)


def equal_width_splitters() -> np.ndarray:
    """Splitters without a model: bucket = the top 12 bits of the key."""
    return (np.arange(1, SPLITTERS + 1, dtype=np.uint64) << np.uint64(52)).astype(np.uint64)


@dataclass
class TrainedModel:
    params: np.ndarray      # float32[NPARAMS]
    norm: np.ndarray        # float32[256] byte-value normalisation
    splitters: np.ndarray   # uint64[SPLITTERS], sorted
    epoch_loss: np.ndarray  # float32[epochs]

    def save(self, path: str) -> None:
        lib = _lib.load()
        check(lib.bwt_model_save(path.encode(), self.params.ctypes.data, self.norm.ctypes.data,
                                 self.splitters.ctypes.data), "bwt_model_save")

    @staticmethod
    def load(path: str) -> "TrainedModel":
        lib = _lib.load()
        p = np.empty(NPARAMS, dtype=np.float32)
        nrm = np.empty(256, dtype=np.float32)
        s = np.empty(SPLITTERS, dtype=np.uint64)
        check(lib.bwt_model_load(path.encode(), p.ctypes.data, nrm.ctypes.data, s.ctypes.data), "bwt_model_load")
        return TrainedModel(p, nrm, s, np.zeros(0, dtype=np.float32))


def _vp(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(int(t.data_ptr()))


def make_samples(workload: datagen.Workload, count: int, seed: int, device: int = 0):
    """(x float32[count][8], t float32[count], norm float32[256]) as CUDA
    tensors from the plain sorter's order of `workload`'s rotations."""
    import torch
    lib = _lib.load()
    buf, off = workload.generate()
    d_in = torch.from_numpy(buf).to(f"cuda:{device}")
    d_norm = torch.empty(256, dtype=torch.float32, device=d_in.device)
    st0 = ctypes.c_void_p(torch.cuda.current_stream(d_in.device).cuda_stream)
    check(lib.bwt_model_byte_norm(_vp(d_in), buf.size, _vp(d_norm), st0), "bwt_model_byte_norm")
    pos = datagen.uniform_ints(seed, count, 0, int(off[-1]) - 1)
    d_pos = torch.from_numpy(pos.view(np.int64)).to(d_in.device)
    d_x = torch.empty((count, 8), dtype=torch.float32, device=d_in.device)
    d_t = torch.empty(count, dtype=torch.float32, device=d_in.device)
    sizes = np.diff(off.astype(np.int64))
    with Plan(max_blocks=workload.num_blocks, max_total_bytes=buf.size, max_block_bytes=int(sizes.max()),
              device=device) as plan:
        st = torch.cuda.current_stream(d_in.device)
        check(lib.bwt_model_samples(plan.handle, _vp(d_in), off.ctypes.data, workload.num_blocks, _vp(d_pos),
                                    count, _vp(d_norm), _vp(d_x), _vp(d_t), ctypes.c_void_p(st.cuda_stream)),
              "bwt_model_samples")
    return d_x, d_t, d_norm


def train(workload: datagen.Workload | None = None, num_samples: int = 1_000_000, epochs: int = 8,
          batch: int = 4096, lr: float = 1e-3, seed: int = 5000, device: int = 0) -> TrainedModel:
    import torch
    lib = _lib.load()
    workload = workload or datagen.learned_train()
    d_x, d_t, d_norm = make_samples(workload, num_samples, seed, device)
    dev = d_x.device
    params = torch.from_numpy(init_params(seed + 1)).to(dev)
    order = np.concatenate([datagen.permutation(seed + 100 + e, num_samples) for e in range(epochs)])
    d_order = torch.from_numpy(order.view(np.int32)).to(dev)
    d_loss = torch.zeros(epochs, dtype=torch.float32, device=dev)
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    check(lib.bwt_model_train(_vp(params), _vp(d_x), _vp(d_t), num_samples, _vp(d_order), epochs, batch,
                              ctypes.c_float(lr), _vp(d_loss), st), "bwt_model_train")
    d_spl = torch.empty(SPLITTERS, dtype=torch.int64, device=dev)
    check(lib.bwt_model_compile(_vp(params), _vp(d_norm), _vp(d_spl), st), "bwt_model_compile")
    torch.cuda.synchronize(dev)
    return TrainedModel(params.cpu().numpy(), d_norm.cpu().numpy(), d_spl.cpu().numpy().view(np.uint64),
                        d_loss.cpu().numpy())


def install(plan: Plan, splitters: np.ndarray) -> None:
    """bwt_plan_set_splitters with a host table."""
    s = np.ascontiguousarray(splitters, dtype=np.uint64)
    check(plan.lib.bwt_plan_set_splitters(plan.handle, s.ctypes.data), "bwt_plan_set_splitters")
