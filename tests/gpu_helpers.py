"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
on a seeded scene and unpack its packed per-pair outputs."""
from dataclasses import dataclass

import numpy as np
import torch

import paper_2508_11790_gb300 as P


@dataclass
class GpuResult:
    plan: "P.Plan"
    off: dict
    xc: np.ndarray       # [P][F][N] complex64
    z_train: np.ndarray  # packed (complex, dequantised for 16-bit storage)
    z_test: np.ndarray
    R: np.ndarray        # packed complex128
    c: np.ndarray        # packed complex64
    info: np.ndarray
    out: np.ndarray      # [pairs][Vte]

    def pair(self, g):
        o = self.off
        W, K = int(o["W"][g]), int(o["K"][g])
        Vte = self.plan.sizes.Vte
        return dict(
            W=W, K=K, start=int(o["start"][g]),
            z_train=self.z_train[o["ztr_off"][g]:o["ztr_off"][g + 1]].reshape(K, W),
            z_test=self.z_test[o["zte_off"][g]:o["zte_off"][g + 1]].reshape(Vte, W),
            R=self.R[o["roff"][g]:o["roff"][g + 1]].reshape(W, W),
            c=self.c[o["woff"][g]:o["woff"][g + 1]],
            a=o["a_tilde"][o["woff"][g]:o["woff"][g + 1]],
            out=self.out[g],
            info=int(self.info[g]),
        )


def ztrain_to_complex(plan, z: torch.Tensor, scale: float = 1.0) -> np.ndarray:
    if plan.precision == P.BS_PREC_FP32:
        return z.cpu().numpy()
    f = z.float().cpu().numpy().reshape(-1, 2) / scale
    return (f[:, 0] + 1j * f[:, 1]).astype(np.complex128)


def run_gpu(cfg, x: np.ndarray, u, precision=P.BS_PREC_FP32, flags=0, keep_xc=True, **plan_kw):
    plan = P.Plan.from_scene_config(cfg, u, precision=precision, flags=flags, **plan_kw)
    b = P.alloc_buffers(plan)
    b.x.copy_(torch.from_numpy(np.ascontiguousarray(x).reshape(-1)))
    P.bs_run(plan, b)
    torch.cuda.synchronize()
    Vte = plan.sizes.Vte
    scale = plan_kw.get("store_scale", 0.0) or 1.0
    res = GpuResult(
        plan=plan, off=plan.offsets(),
        xc=b.xc.cpu().numpy().reshape(cfg.P, -1, cfg.N) if keep_xc else None,
        z_train=ztrain_to_complex(plan, b.z_train, scale),
        z_test=b.z_test.cpu().numpy(),
        R=b.R.cpu().numpy(), c=b.c.cpu().numpy(), info=b.info.cpu().numpy(),
        out=b.out.cpu().numpy()[: plan.sizes.pairs * Vte].reshape(plan.sizes.pairs, Vte),
    )
    del b
    return res


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)
