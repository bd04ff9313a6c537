"""Many beams of different grid sizes marched together in one persistent CUDA
launch per call (include/nlse.h, nlse_batch_*), optionally replayed from a
captured CUDA graph.  FP32 fields, n = 256..4096."""
from __future__ import annotations

import numpy as np
import torch

from . import capi
from .grid import _aligned_workspace, make_params


class Batch:
    def __init__(self, cfgs: list, tuning: dict | None = None, device=None,
                 stream: torch.cuda.Stream | None = None):
        self.cfgs = cfgs
        self.params = [make_params(c, "fp32", 0) for c in cfgs]
        self.ns = [int(c["n"]) for c in cfgs]
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        t = None
        if tuning is not None:
            t = capi.nlse_batch_tuning()
            t.threads = int(tuning.get("threads", 256))
            t.ctas_per_sm = int(tuning.get("ctas_per_sm", 0))
            t.timeout_ms = int(tuning.get("timeout_ms", 2000))
            t.debug_skip_item = int(tuning.get("debug_skip_item", -1))
            t.radix = int(tuning.get("radix", 16))
            t.per_thread_columns = int(tuning.get("per_thread_columns", 0))
        self.ws_bytes = capi.nlse_batch_workspace_size(self.params)
        self._ws, ptr = _aligned_workspace(self.ws_bytes, self.device)
        self.h = capi.nlse_batch_create(self.params, t, self.stream.cuda_stream, ptr, self.ws_bytes)

    def load(self, beam: int, U) -> "Batch":
        if isinstance(U, torch.Tensor) and U.is_cuda:
            u = U.to(torch.complex64).contiguous()
            capi.nlse_batch_load_field(self.h, beam, u.data_ptr(), True)
            self.stream.synchronize()
        else:
            a = np.ascontiguousarray(U, dtype=np.complex64)
            assert a.shape == (self.ns[beam], self.ns[beam])
            capi.nlse_batch_load_field(self.h, beam, a.ctypes.data, False)
        return self

    def step(self, nsteps: int) -> "Batch":
        capi.nlse_batch_step(self.h, nsteps)
        return self

    def capture(self, nsteps: int) -> "Batch":
        capi.nlse_batch_capture(self.h, nsteps)
        return self

    def replay(self) -> "Batch":
        capi.nlse_batch_replay(self.h)
        return self

    def status(self) -> int:
        return capi.nlse_batch_status(self.h)

    @property
    def steps_taken(self) -> int:
        return capi.nlse_batch_steps_taken(self.h)

    def field(self, beam: int, device: bool = False):
        n = self.ns[beam]
        if device:
            out = torch.empty((n, n), dtype=torch.complex64, device=self.device)
            capi.nlse_batch_read_field(self.h, beam, out.data_ptr(), True)
            return out
        out = np.empty((n, n), dtype=np.complex64)
        capi.nlse_batch_read_field(self.h, beam, out.ctypes.data, False)
        return out

    def power(self, beam: int) -> float:
        return capi.nlse_batch_power(self.h, beam)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            capi.nlse_batch_destroy(self.h)
            self.h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
