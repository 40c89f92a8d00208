"""Unfused comparison form: the same grouped M-rPIE schedule written with
stock PyTorch ops and cuFFT (torch.fft), one op per step, as a framework
user would write it.  It is NOT the product path and shares no kernels with
libpty; it exists only so that the fused sm_103a path can be timed against
the straightforward GPU implementation on the same GPU and inputs.

Per group of disjoint crop boxes (processed in chunks), exactly the readings
of the library: unitary 2-D DFT, Psi' = sqrt(I) Psi / (sqrt(S) + eps), the
object update of Eq. 6 with the group's Pmax, and the probe update of Eq. 5
as the ratio of the group's summed numerators and denominators.
"""
import torch


class UnfusedRPIE:
    def __init__(self, O0, P0, I_u16, pos, W, max_chunk=64):
        dev = O0.device
        self.O = O0.clone()
        self.P = P0.clone()
        self.W = W
        self.Ish = torch.fft.ifftshift(I_u16.to(torch.float32), dim=(-2, -1)).sqrt_()
        self.sumI = float(I_u16.to(torch.float64).sum())
        corners = torch.floor(pos.double() + 0.5).long()
        self.corners = corners
        from .pty import group_positions
        self.groups = [torch.as_tensor(g, dtype=torch.long, device=dev)
                       for g in group_positions(pos.cpu().numpy(), W)]
        self.max_chunk = max_chunk
        ar = torch.arange(W, device=dev)
        self.ar = ar

    def _rows_cols(self, idx):
        c = self.corners[idx]
        rows = (c[:, 0, None] + self.ar[None, :])[:, :, None]
        cols = (c[:, 1, None] + self.ar[None, :])[:, None, :]
        return rows, cols

    def iteration(self, alpha_O=1.0, alpha_P=1.0, beta=1.0, gamma=0.1, eps=1.0, reg_eps=1e-12):
        err = torch.zeros((), dtype=torch.float64, device=self.O.device)
        for g in self.groups:
            Pint = (self.P.real ** 2 + self.P.imag ** 2).sum(0)
            Pmax = Pint.max()
            obj_den = gamma * Pmax + (1 - gamma) * Pint + reg_eps * Pmax
            num = torch.zeros_like(self.P)
            den = torch.zeros_like(Pint)
            osum = torch.zeros((), device=self.O.device)
            for s in range(0, len(g), self.max_chunk):
                idx = g[s:s + self.max_chunk]
                rows, cols = self._rows_cols(idx)
                o = self.O[rows, cols]                                   # gather crops
                psi = self.P[None] * o[:, None]                          # exit waves
                Psi = torch.fft.fft2(psi, norm="ortho")                 # cuFFT
                S = (Psi.real ** 2 + Psi.imag ** 2).sum(1)
                sqI = self.Ish[idx]
                a = S.sqrt()
                err += ((a - sqI) ** 2).sum(dtype=torch.float64)
                Psi = Psi * (sqI / (a + eps))[:, None]
                D = torch.fft.ifft2(Psi, norm="ortho") - psi
                upd = (D * self.P.conj()[None]).sum(1)
                self.O[rows, cols] = o + alpha_O * upd / obj_den        # scatter back
                num += (D * o.conj()[:, None]).sum(0)
                a2 = o.real ** 2 + o.imag ** 2
                om = a2.amax(dim=(-2, -1))
                den += (beta * om[:, None, None] + (1 - beta) * a2).sum(0)
                osum += om.sum()
            self.P += alpha_P * num / (den + reg_eps * osum)[None]
        return float(err) / self.sumI
