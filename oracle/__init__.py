"""Oracle for the pseudopotential D2Q9 lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: a plain, slow, obviously correct CPU reference in
float64, written from the paper (Czelusniak, Mapelli, Cabezas Gomez, Wagner,
"Shaping the equation of state to improve numerical accuracy and stability of
the pseudopotential lattice Boltzmann method"). Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` legs may import it. It shares no code with the CUDA
library under ``paper_2107_06355_gb300/`` and never imports it.

Modules:
  eos  -- Carnahan-Starling EOS, Maxwell rule, Smooth C-S shaping, epsilon/sigma.
  lbm  -- one time step of the D2Q9 MRT lattice Boltzmann equation with the
          Shan-Chen force and the Guo / Li forcing schemes, and the optional
          surface-tension control the paper's Sec. V names (Li & Luo 2013).
"""
