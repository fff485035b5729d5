"""CPU oracle of the QIEO generation loop (test infrastructure; see qieo_oracle.c)."""
